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

#include <type_traits>

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

// One sub-stage with every twiddle read from the length-M table: entry offset
// JP < SIG of the sub-stage takes (w_{L_s}^p w_{SIG RHO}^JP)^q = w_M^(q B),
// B = TS p + JP M / (SIG RHO), for q = 1 .. RHO-1 (q B < M).  FP64 passes are
// bound by the FP64 pipe, so table loads replace the complex products that
// substage_jp spends on forming the powers (a fifth of their twiddle work).
// FP32 passes keep substage_jp: they are bound by instruction issue and load
// latency, and the table loads made the M = 4374 last-axis pass 145 -> 170 us.
template <int SIGN, bool DIT, int RHO, int SIG, int RG, int JP, int TS, int M, typename C>
__device__ __forceinline__ void substage_tab(C* v, int p, const C* __restrict__ tw) {
  const int b = TS * p + JP * (M / (SIG * RHO));
  C tq[RHO];
#pragma unroll
  for (int q = 1; q < RHO; ++q) tq[q] = __ldg(&tw[q * b]);
#pragma unroll
  for (int jb = 0; jb < RG / (SIG * RHO); ++jb) {
    C e[RHO];
#pragma unroll
    for (int q = 0; q < RHO; ++q) e[q] = v[jb * SIG * RHO + JP + q * SIG];
    if constexpr (DIT) {
#pragma unroll
      for (int q = 1; q < RHO; ++q) e[q] = twmul<SIGN>(e[q], tq[q]);
    }
    dft_small<SIGN, RHO>(e);
    if constexpr (!DIT) {
#pragma unroll
      for (int q = 1; q < RHO; ++q) e[q] = twmul<SIGN>(e[q], tq[q]);
    }
#pragma unroll
    for (int q = 0; q < RHO; ++q) v[jb * SIG * RHO + JP + q * SIG] = e[q];
  }
  if constexpr (JP + 1 < SIG) substage_tab<SIGN, DIT, RHO, SIG, RG, JP + 1, TS, M>(v, p, tw);
}

template <int SIGN, bool DIT, bool FIRST, int RHO, int SIG, int RG, int TS, int M, typename C>
__device__ __forceinline__ void ct_substage(C* v, int p, const C* __restrict__ tw) {
  if constexpr (FIRST) {
    substage_const<SIGN, DIT, RHO, SIG, RG, 0>(v);
  } else if constexpr (sizeof(C) == 16) {
    substage_tab<SIGN, DIT, RHO, SIG, RG, 0, TS, M>(v, p, tw);
  } else {
    const C wb = __ldg(&tw[p * TS]);   // w_{L_s}^p
    substage_jp<SIGN, DIT, RHO, SIG, RG, 0>(v, wb);
  }
}

// Natural index of the entries of the first pass (L_{t-1} = 1).  Its unit b
// holds positions b RG + j, j = d1 + RA d2 + RA RB d3, which carry the input
// (DIT) or output (DIF) index
//     n = rest(b) + (M / RG) (d1 RB RC + d2 RC + d3),
// rest(b) = the remaining position digits of b, each weighted by the product of
// the radices of the stages after its own.
template <int RA, int RB, int RC>
__host__ __device__ constexpr int ct_revj(int j) {
  return (j % RA) * RB * RC + ((j / RA) % RB) * RC + j / (RA * RB);
}
__host__ __device__ constexpr int ct_weight(int M, int t) {   // product of the radices after stage t
  int w = 1;
  for (int u = t + 1; u < ct_plan(M).nst; ++u) w *= ct_plan(M).R[u];
  return w;
}
template <int M, int T>
__device__ __forceinline__ int ct_rest_from(int b) {
  constexpr CtPlan P = ct_plan(M);
  if constexpr (T >= P.nst) {
    return 0;
  } else {
    constexpr int R = P.R[T];
    constexpr int W = ct_weight(M, T);
    return (b % R) * W + ct_rest_from<M, T + 1>(b / R);
  }
}
template <int M>
__device__ __forceinline__ int ct_rest(int b) {
  constexpr CtPlan P = ct_plan(M);
  constexpr int s0 = (P.ra[0] > 1) + (P.rb[0] > 1) + (P.rc[0] > 1);
  return ct_rest_from<M, s0>(b);
}
// Placeholder for "read from / write to the shared buffer".
struct CtBuf {};

// Sources with a member kWriteBack = true also get write_back(line, n, value)
// for every entry, called after all of a unit's entries have been read.
template <typename S, typename = void>
struct ct_writes_back : std::false_type {};
template <typename S>
struct ct_writes_back<S, std::void_t<decltype(S::kWriteBack)>> : std::integral_constant<bool, S::kWriteBack> {};

// Sources with a member kRanged = true are called as src.ranged(line, nb, n0,
// span) for input n = nb + n0, where n0 and span are compile-time constants of
// the pass and 0 <= nb < span: a source whose entries depend on where n lies
// (zero padding, a mirrored half) can then decide for the whole range
// [n0, n0 + span) with a test that is the same in every thread.
template <typename S, typename = void>
struct ct_ranged : std::false_type {};
template <typename S>
struct ct_ranged<S, std::void_t<decltype(S::kRanged)>> : std::integral_constant<bool, S::kRanged> {};

// One pass: butterflies of radix RA RB RC on stride LP, NT threads, NL lines
// interleaved (element (m, line) at m NL + line, no padding).  The first pass
// may take its entries from a source instead of the buffer (DIT: src(line, n)
// returns input n, so the caller's scatter into digit-reversed order and its
// zero padding disappear) and may hand its results to a sink instead of the
// buffer (DIF: snk(line, n, value) receives output n).
template <int SIGN, bool DIT, int NL, int NT, int M, int LP, int RA, int RB, int RC, typename C,
          typename Src = CtBuf, typename Snk = CtBuf>
__device__ __forceinline__ void ct_pass(C* buf, const C* __restrict__ tw, const Src& src = Src(),
                                        const Snk& snk = Snk()) {
  constexpr int RG = RA * RB * RC;
  constexpr int units = M / RG;
  constexpr int total = units * NL;
  constexpr int tsA = M / (LP * RA);
  constexpr int tsB = tsA / RB;
  constexpr int tsC = tsB / RC;
  constexpr int step = LP * NL;
  constexpr bool FIRST = (LP == 1);
  constexpr bool FROM_SRC = !std::is_same<Src, CtBuf>::value;
  constexpr bool TO_SNK = !std::is_same<Snk, CtBuf>::value;
  static_assert(FIRST || (!FROM_SRC && !TO_SNK), "sources and sinks belong to the first pass");
#pragma unroll 1
  for (int u = threadIdx.x; u < total; u += NT) {
    const int line = (NL == 1) ? 0 : u % NL;
    const int unit = (NL == 1) ? u : u / NL;
    const int b = unit / LP;
    const int p = unit - b * LP;
    C* base = buf + (b * LP * RG + p) * NL + line;
    int nb = 0;
    if constexpr (FROM_SRC || TO_SNK) nb = ct_rest<M>(b);
    C v[RG];
#pragma unroll
    for (int j = 0; j < RG; ++j) {
      if constexpr (FROM_SRC && ct_ranged<Src>::value) v[j] = src.ranged(line, nb, (M / RG) * ct_revj<RA, RB, RC>(j), M / RG);
      else if constexpr (FROM_SRC) v[j] = src(line, nb + (M / RG) * ct_revj<RA, RB, RC>(j));
      else v[j] = base[j * step];
    }
    if constexpr (FROM_SRC && ct_writes_back<Src>::value) {
      // a source that also stores what it produced does so after all its loads
#pragma unroll
      for (int j = 0; j < RG; ++j) src.write_back(line, nb + (M / RG) * ct_revj<RA, RB, RC>(j), v[j]);
    }
    if constexpr (DIT) {
      ct_substage<SIGN, DIT, FIRST, RA, 1, RG, tsA, M>(v, p, tw);
      if constexpr (RB > 1) ct_substage<SIGN, DIT, FIRST, RB, RA, RG, tsB, M>(v, p, tw);
      if constexpr (RC > 1) ct_substage<SIGN, DIT, FIRST, RC, RA * RB, RG, tsC, M>(v, p, tw);
    } else {
      if constexpr (RC > 1) ct_substage<SIGN, DIT, FIRST, RC, RA * RB, RG, tsC, M>(v, p, tw);
      if constexpr (RB > 1) ct_substage<SIGN, DIT, FIRST, RB, RA, RG, tsB, M>(v, p, tw);
      ct_substage<SIGN, DIT, FIRST, RA, 1, RG, tsA, M>(v, p, tw);
    }
#pragma unroll
    for (int j = 0; j < RG; ++j) {
      if constexpr (TO_SNK) snk(line, nb + (M / RG) * ct_revj<RA, RB, RC>(j), v[j]);
      else base[j * step] = v[j];
    }
  }
}

// Decimation-in-time passes I .. HI-1 (HI < 0: through the last pass).
template <int SIGN, int NL, int NT, int M, int I, int HI = -1, typename C>
__device__ __forceinline__ void ct_dit_from(C* buf, const C* __restrict__ tw) {
  constexpr CtPlan P = ct_plan(M);
  constexpr int E = HI < 0 ? P.npass : HI;
  if constexpr (I < E) {
    ct_pass<SIGN, true, NL, NT, M, P.lp[I], P.ra[I], P.rb[I], P.rc[I]>(buf, tw);
    __syncthreads();
    ct_dit_from<SIGN, NL, NT, M, I + 1, HI>(buf, tw);
  }
}

template <int SIGN, int NL, int NT, int M, int I, int LO = 0, typename C>
__device__ __forceinline__ void ct_dif_from(C* buf, const C* __restrict__ tw) {
  constexpr CtPlan P = ct_plan(M);
  if constexpr (I >= LO) {
    ct_pass<SIGN, false, NL, NT, M, P.lp[I], P.ra[I], P.rb[I], P.rc[I]>(buf, tw);
    __syncthreads();
    ct_dif_from<SIGN, NL, NT, M, I - 1, LO>(buf, tw);
  }
}

// Decimation in time: digit-reversed input (ct_perm order) -> natural output.
// The caller must __syncthreads() after filling buf; ends with a barrier.
template <int SIGN, int NL, int NT, int M, typename C>
__device__ __forceinline__ void fft_dit_ct(C* buf, const C* __restrict__ tw) {
  static_assert(ct_plan(M).ok, "transform length must factor into 2, 3, 4, 5");
  ct_dit_from<SIGN, NL, NT, M, 0>(buf, tw);
}

// The same with the input read from src(line, n), n the natural index (no
// scatter into buf beforehand; the first pass reads src and writes buf).
template <int SIGN, int NL, int NT, int M, typename C, typename Src>
__device__ __forceinline__ void fft_dit_ct_src(C* buf, const C* __restrict__ tw, const Src& src) {
  constexpr CtPlan P = ct_plan(M);
  static_assert(P.ok, "transform length must factor into 2, 3, 4, 5");
  ct_pass<SIGN, true, NL, NT, M, 1, P.ra[0], P.rb[0], P.rc[0]>(buf, tw, src);
  __syncthreads();
  ct_dit_from<SIGN, NL, NT, M, 1>(buf, tw);
}

// Decimation in frequency: natural input -> digit-reversed output.
template <int SIGN, int NL, int NT, int M, typename C>
__device__ __forceinline__ void fft_dif_ct(C* buf, const C* __restrict__ tw) {
  static_assert(ct_plan(M).ok, "transform length must factor into 2, 3, 4, 5");
  ct_dif_from<SIGN, NL, NT, M, ct_plan(M).npass - 1>(buf, tw);
}

// Inverse transform of each line (decimation in time, input from src in the
// first pass), pointwise scaling, forward transform (decimation in frequency).
// The inverse's last pass and the forward's first pass act on the same
// entries p + j LP of the natural order (b = 0 in both), so one thread does
// both in registers with mul(line, m, v) in between: one shared-memory round
// trip and one barrier fewer per line.  Hooks: after_first() once the
// inverse's first pass is done in every thread (src is no longer read);
// before_fused() ahead of the fused pass (mul's data must be in place);
// after_fused() once the fused pass is done in every thread.  Needs two
// passes at least; ends with a barrier.
template <int SIGN_I, int SIGN_F, int NL, int NT, int M, typename C, typename Src, typename Mul, typename H1,
          typename H2, typename H3>
__device__ __forceinline__ void ct_inverse_scale_forward(C* buf, const C* __restrict__ tw, const Src& src,
                                                         const Mul& mul, const H1& after_first,
                                                         const H2& before_fused, const H3& after_fused) {
  constexpr CtPlan P = ct_plan(M);
  static_assert(P.ok && P.npass >= 2, "the fused pass needs a transform of two passes at least");
  constexpr int I = P.npass - 1;
  constexpr int LP = P.lp[I], RA = P.ra[I], RB = P.rb[I], RC = P.rc[I];
  constexpr int RG = RA * RB * RC;
  static_assert(LP * RG == M, "the last pass spans the line");
  constexpr int tsA = M / (LP * RA);
  constexpr int tsB = tsA / RB;
  constexpr int tsC = tsB / RC;
  constexpr int step = LP * NL;
  ct_pass<SIGN_I, true, NL, NT, M, 1, P.ra[0], P.rb[0], P.rc[0]>(buf, tw, src);
  __syncthreads();
  after_first();
  ct_dit_from<SIGN_I, NL, NT, M, 1, I>(buf, tw);
  before_fused();
#pragma unroll 1
  for (int u = threadIdx.x; u < LP * NL; u += NT) {
    const int line = (NL == 1) ? 0 : u % NL;
    const int p = (NL == 1) ? u : u / NL;
    C* base = buf + p * NL + line;
    C v[RG];
#pragma unroll
    for (int j = 0; j < RG; ++j) v[j] = base[j * step];
    ct_substage<SIGN_I, true, false, RA, 1, RG, tsA, M>(v, p, tw);
    if constexpr (RB > 1) ct_substage<SIGN_I, true, false, RB, RA, RG, tsB, M>(v, p, tw);
    if constexpr (RC > 1) ct_substage<SIGN_I, true, false, RC, RA * RB, RG, tsC, M>(v, p, tw);
#pragma unroll
    for (int j = 0; j < RG; ++j) v[j] = mul(line, p + j * LP, v[j]);
    if constexpr (RC > 1) ct_substage<SIGN_F, false, false, RC, RA * RB, RG, tsC, M>(v, p, tw);
    if constexpr (RB > 1) ct_substage<SIGN_F, false, false, RB, RA, RG, tsB, M>(v, p, tw);
    ct_substage<SIGN_F, false, false, RA, 1, RG, tsA, M>(v, p, tw);
#pragma unroll
    for (int j = 0; j < RG; ++j) base[j * step] = v[j];
  }
  __syncthreads();
  after_fused();
  ct_dif_from<SIGN_F, NL, NT, M, I - 1>(buf, tw);
}

// The same with every output handed to snk(line, n, value), n the natural
// index, instead of being stored (the last pass reads buf and calls snk; buf
// is left partly overwritten).  Ends without a barrier.
template <int SIGN, int NL, int NT, int M, typename C, typename Snk>
__device__ __forceinline__ void fft_dif_ct_snk(C* buf, const C* __restrict__ tw, const Snk& snk) {
  constexpr CtPlan P = ct_plan(M);
  static_assert(P.ok, "transform length must factor into 2, 3, 4, 5");
  ct_dif_from<SIGN, NL, NT, M, P.npass - 1, 1>(buf, tw);
  ct_pass<SIGN, false, NL, NT, M, 1, P.ra[0], P.rb[0], P.rc[0], C, CtBuf, Snk>(buf, tw, CtBuf(), snk);
}

}  // namespace ghb
