// Size-specialised shared-memory FFT: the same decimation-in-time /
// decimation-in-frequency stages as fft.cuh, for a transform length M known at
// compile time.
//
// With M fixed, every pass's radices, stride L_{t-1}, unit count and twiddle
// step are constants, so a butterfly's shared-memory operands sit at constant
// offsets from one base address and the index arithmetic of the runtime plan
// (division by L_{t-1}, padded indices) disappears.  The stages are ordered
// with the odd radices first (5s, then 3s, then 4s and 2s): the first pass,
// whose butterflies read R_1 R_2 R_3 consecutive entries, then has an odd
// stride between neighbouring threads and reaches all shared-memory banks
// without padding, and later passes read consecutive entries across a warp.
// The stages of a pass run in registers (up to three, radix product <= 32).
// Inside the first pass every twiddle is a root of unity that the compiler
// evaluates.
//
// The digit-reversal permutation follows this stage order, so callers use the
// table built by ct_perm (not the runtime plan's).
#pragma once

#include "fft.cuh"

namespace ghb {

constexpr int kCtMaxStages = 24;
constexpr int kCtMaxPasses = 12;

struct CtPlan {
  int M;
  int nst;                 // number of stages
  int R[kCtMaxStages];     // stage radices in DIT order
  int npass;
  int ra[kCtMaxPasses];    // radices of pass i in DIT order (1 = absent)
  int rb[kCtMaxPasses];
  int rc[kCtMaxPasses];
  int lp[kCtMaxPasses];    // product of the radices of the earlier passes
  bool ok;                 // M factors into 2, 3, 4, 5
};

__host__ __device__ constexpr CtPlan ct_plan(int M) {
  CtPlan p{};
  p.M = M;
  int m = M, n = 0;
  while (m % 5 == 0 && n < kCtMaxStages) { p.R[n++] = 5; m /= 5; }
  while (m % 3 == 0 && n < kCtMaxStages) { p.R[n++] = 3; m /= 3; }
  while (m % 4 == 0 && n < kCtMaxStages) { p.R[n++] = 4; m /= 4; }
  while (m % 2 == 0 && n < kCtMaxStages) { p.R[n++] = 2; m /= 2; }
  p.nst = n;
  p.ok = (m == 1) && M > 1;
  int t = 0, L = 1, np = 0;
  while (t < n && np < kCtMaxPasses) {
    int r[3] = {1, 1, 1};
    int k = 0, prod = 1;
    while (k < 3 && t < n && prod * p.R[t] <= 32) {
      r[k] = p.R[t];
      prod *= p.R[t];
      ++k;
      ++t;
    }
    p.ra[np] = r[0];
    p.rb[np] = r[1];
    p.rc[np] = r[2];
    p.lp[np] = L;
    L *= prod;
    ++np;
  }
  p.npass = np;
  p.ok = p.ok && t == n;
  return p;
}

// perm[n]: write n in mixed radix with the last stage's radix least significant;
// the position has the digits in stage order, first stage least significant.
inline void ct_perm(int M, int* perm) {
  const CtPlan p = ct_plan(M);
  for (int n = 0; n < M; ++n) {
    int rem = n, pos = 0;
    int q[kCtMaxStages] = {0};
    for (int t = p.nst - 1; t >= 0; --t) {
      q[t] = rem % p.R[t];
      rem /= p.R[t];
    }
    int L = 1;
    for (int t = 0; t < p.nst; ++t) {
      pos += q[t] * L;
      L *= p.R[t];
    }
    perm[n] = pos;
  }
}

// One sub-stage of a pass whose every butterfly has p = 0 (the first pass,
// L_{t-1} = 1): all twiddles are the compile-time roots w_{SIG RHO}^{JP q}.
template <int SIGN, bool DIT, int RHO, int SIG, int RG, int JP, typename C>
__device__ __forceinline__ void substage_const(C* v) {
  using R = decltype(v[0].x);
#pragma unroll
  for (int jb = 0; jb < RG / (SIG * RHO); ++jb) {
    C e[RHO];
#pragma unroll
    for (int q = 0; q < RHO; ++q) e[q] = v[jb * SIG * RHO + JP + q * SIG];
    if constexpr (DIT && JP > 0) {
#pragma unroll
      for (int q = 1; q < RHO; ++q)
        e[q] = twmul<SIGN>(e[q], mk(R(root_cos(JP * q, SIG * RHO)), R(-root_sin(JP * q, SIG * RHO))));
    }
    dft_small<SIGN, RHO>(e);
    if constexpr (!DIT && JP > 0) {
#pragma unroll
      for (int q = 1; q < RHO; ++q)
        e[q] = twmul<SIGN>(e[q], mk(R(root_cos(JP * q, SIG * RHO)), R(-root_sin(JP * q, SIG * RHO))));
    }
#pragma unroll
    for (int q = 0; q < RHO; ++q) v[jb * SIG * RHO + JP + q * SIG] = e[q];
  }
  if constexpr (JP + 1 < SIG) substage_const<SIGN, DIT, RHO, SIG, RG, JP + 1>(v);
}

template <int SIGN, bool DIT, bool FIRST, int RHO, int SIG, int RG, int TS, typename C>
__device__ __forceinline__ void ct_substage(C* v, int p, const C* __restrict__ tw) {
  if constexpr (FIRST) {
    substage_const<SIGN, DIT, RHO, SIG, RG, 0>(v);
  } else {
    const C wb = __ldg(&tw[p * TS]);   // w_{L_s}^p
    substage_jp<SIGN, DIT, RHO, SIG, RG, 0>(v, wb);
  }
}

// One pass: butterflies of radix RA RB RC on stride LP, NT threads, NL lines
// interleaved (element (m, line) at m NL + line, no padding).
template <int SIGN, bool DIT, int NL, int NT, int M, int LP, int RA, int RB, int RC, typename C>
__device__ __forceinline__ void ct_pass(C* buf, const C* __restrict__ tw) {
  constexpr int RG = RA * RB * RC;
  constexpr int units = M / RG;
  constexpr int total = units * NL;
  constexpr int tsA = M / (LP * RA);
  constexpr int tsB = tsA / RB;
  constexpr int tsC = tsB / RC;
  constexpr int step = LP * NL;
  constexpr bool FIRST = (LP == 1);
#pragma unroll 1
  for (int u = threadIdx.x; u < total; u += NT) {
    const int line = (NL == 1) ? 0 : u % NL;
    const int unit = (NL == 1) ? u : u / NL;
    const int b = unit / LP;
    const int p = unit - b * LP;
    C* base = buf + (b * LP * RG + p) * NL + line;
    C v[RG];
#pragma unroll
    for (int j = 0; j < RG; ++j) v[j] = base[j * step];
    if constexpr (DIT) {
      ct_substage<SIGN, DIT, FIRST, RA, 1, RG, tsA>(v, p, tw);
      if constexpr (RB > 1) ct_substage<SIGN, DIT, FIRST, RB, RA, RG, tsB>(v, p, tw);
      if constexpr (RC > 1) ct_substage<SIGN, DIT, FIRST, RC, RA * RB, RG, tsC>(v, p, tw);
    } else {
      if constexpr (RC > 1) ct_substage<SIGN, DIT, FIRST, RC, RA * RB, RG, tsC>(v, p, tw);
      if constexpr (RB > 1) ct_substage<SIGN, DIT, FIRST, RB, RA, RG, tsB>(v, p, tw);
      ct_substage<SIGN, DIT, FIRST, RA, 1, RG, tsA>(v, p, tw);
    }
#pragma unroll
    for (int j = 0; j < RG; ++j) base[j * step] = v[j];
  }
}

template <int SIGN, int NL, int NT, int M, int I, typename C>
__device__ __forceinline__ void ct_dit_from(C* buf, const C* __restrict__ tw) {
  constexpr CtPlan P = ct_plan(M);
  if constexpr (I < P.npass) {
    ct_pass<SIGN, true, NL, NT, M, P.lp[I], P.ra[I], P.rb[I], P.rc[I]>(buf, tw);
    __syncthreads();
    ct_dit_from<SIGN, NL, NT, M, I + 1>(buf, tw);
  }
}

template <int SIGN, int NL, int NT, int M, int I, typename C>
__device__ __forceinline__ void ct_dif_from(C* buf, const C* __restrict__ tw) {
  constexpr CtPlan P = ct_plan(M);
  if constexpr (I >= 0) {
    ct_pass<SIGN, false, NL, NT, M, P.lp[I], P.ra[I], P.rb[I], P.rc[I]>(buf, tw);
    __syncthreads();
    ct_dif_from<SIGN, NL, NT, M, I - 1>(buf, tw);
  }
}

// Decimation in time: digit-reversed input (ct_perm order) -> natural output.
// The caller must __syncthreads() after filling buf; ends with a barrier.
template <int SIGN, int NL, int NT, int M, typename C>
__device__ __forceinline__ void fft_dit_ct(C* buf, const C* __restrict__ tw) {
  static_assert(ct_plan(M).ok, "transform length must factor into 2, 3, 4, 5");
  ct_dit_from<SIGN, NL, NT, M, 0>(buf, tw);
}

// Decimation in frequency: natural input -> digit-reversed output.
template <int SIGN, int NL, int NT, int M, typename C>
__device__ __forceinline__ void fft_dif_ct(C* buf, const C* __restrict__ tw) {
  static_assert(ct_plan(M).ok, "transform length must factor into 2, 3, 4, 5");
  ct_dif_from<SIGN, NL, NT, M, ct_plan(M).npass - 1>(buf, tw);
}

}  // namespace ghb
