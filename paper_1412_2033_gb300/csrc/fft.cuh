// Shared-memory mixed-radix FFT for sm_103a.
//
// The double-grid operator of the Ga scheme (Algorithm 2; Lemma integ_eval_VM)
// needs DFTs of length M along each axis, where M >= 2N-1 is any size whose
// prime factors are <= 31 (5-smooth by default, e.g. M = 2*3^7 = 4374).
// Convention (eq. DFT_coef, eq. DFT): the inverse DFT is
//     u[m] = sum_k x[k] exp(+2 pi i m k / M)          (SIGN = +1, unscaled)
// and the forward DFT is
//     X[k] = sum_m u[m] exp(-2 pi i m k / M)          (SIGN = -1; the 1/M
// factor is applied by the caller when it truncates to Z_N).
//
// Data layout in shared memory: NL independent lines interleaved,
// element (m, line) at padded index pad(m * NL + line), so that consecutive
// threads touch consecutive words and strided butterflies spread over banks.
//
// Algorithm (in place, one shared buffer).  M = R_1 ... R_s (radices 2,3,4,5 or
// a prime <= 31).  Decimation in time (DIT) takes digit-reversed input (the
// caller scatters x[n] to position perm[n]) and returns natural order; stage t
// combines R_t transforms of length L_{t-1} = R_1...R_{t-1}: for block b and
// position p < L_{t-1} the butterfly reads the R_t entries b L_t + p + q L_{t-1},
// multiplies entry q by w_{L_t}^{pq}, applies DFT_{R_t} and writes back.
// Decimation in frequency (DIF) runs the same stages in reverse order with the
// twiddle after the small DFT: natural input, digit-reversed output (X[k] at
// perm[k]).  A line therefore goes inverse (DIT) -> pointwise multiply ->
// forward (DIF) without any permutation pass.
//
// Register blocking: consecutive stages are grouped into passes of at most
// three stages (radix product <= 32).  The stages of a group act inside the
// sets {b L_g + p + j L_{t-1} : j < R_g}, so one thread loads such a set into
// registers, runs the group's stages there and writes it back: one shared-memory
// round trip and one barrier per pass instead of per stage.  Twiddles: the
// stage-s factor w_{L_s}^{(p + j' L_{t-1}) q} = (w_{L_s}^p w_{sigma rho}^{j'})^q is a
// table load per pass and sub-stage (w_{L_s}^p) times a root of unity of small
// order that the compiler evaluates, raised to the power q by multiplication.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace ghb {

constexpr int kMaxStages = 24;
constexpr int kMaxPasses = 24;
constexpr int kMaxGenericRadix = 31;

// Division by an invariant 32-bit integer with a multiply-high (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// round-up variant): q = (t + ((n - t) >> 1)) >> (l - 1), t = umulhi(n, m),
// m = floor(2^32 (2^l - d) / d) + 1, l = ceil(log2 d).  Exact for every 32-bit n.
struct FastDiv {
  unsigned d;
  unsigned m;
  int l;
};

inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  int l = 0;
  while ((1ull << l) < d) ++l;
  f.l = l;
  if (d == 1) {
    f.m = 0;
  } else {
    const unsigned long long num = (1ull << 32) * ((1ull << l) - d);
    f.m = static_cast<unsigned>(num / d + 1);
  }
  return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
  if (f.d == 1) return n;
  const unsigned t = __umulhi(n, f.m);
  return (t + ((n - t) >> 1)) >> (f.l - 1);
}

// Shapes of one pass: the radices of its stages in DIT order.
enum PassShape {
  SH_2 = 0, SH_3, SH_4, SH_5,
  SH_2_3, SH_3_3, SH_2_5, SH_4_3, SH_3_5, SH_4_4, SH_4_5, SH_5_5, SH_4_2,
  SH_2_3_3, SH_3_3_3, SH_4_2_3, SH_2_3_5, SH_4_4_2,
  SH_GENERIC,   // one stage of a prime radix 7..31 (O(R^2) definition)
  SH_COUNT
};

// Plan of one length-M transform.  Tables live in device memory.
struct FftPlan {
  int M;
  int nst;                   // number of stages
  int R[kMaxStages];         // radix of DIT stage t
  int Lp[kMaxStages];        // L_{t-1}: product of the radices before stage t
  // passes per precision ([0] FP64: at most 18 entries per thread so the
  // registers hold them; [1] FP32: at most 32)
  int npass[2];
  int pshape[2][kMaxPasses];    // PassShape of each pass (DIT order)
  int pR[2][kMaxPasses];        // radix product of the pass (or the prime)
  int pLp[2][kMaxPasses];       // L_{t-1} of its first stage
  FastDiv pdiv[2][kMaxPasses];  // division by pLp
  const int* perm;           // perm[n]: digit-reversed position of index n
  const int* perm_ct;        // the same for the stage order of fft_ct.cuh (null if M has no
                             // size-specialised kernels)
  const double2* tw64;       // tw64[j] = exp(-2 pi i j / M)
  const float2* tw32;        // the same rounded to float
  // launch configuration chosen by the autotuner (host-side choices; 0 = size rule)
  int tile[2];               // column-pass tile width ([0] FP64, [1] FP32)
  int rows32;                // rows per CTA of the FP32 2-D operator's last-axis pass
  int ct_col, ct_row;        // 1: size-specialised FP32 kernels for the column / last-axis passes
};

template <typename T> struct CT;
template <> struct CT<double> { using type = double2; };
template <> struct CT<float> { using type = float2; };

__device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return mk(s * a.x, s * a.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return mk(s * a.x, s * a.y); }

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// a * w (SIGN = -1) or a * conj(w) (SIGN = +1); w in the forward convention.
template <int SIGN, typename C>
__device__ __forceinline__ C twmul(C a, C w) {
  if (SIGN < 0) return mk(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
  return mk(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}

// i * SIGN * a
template <int SIGN, typename C>
__device__ __forceinline__ C rot(C a) {
  return SIGN > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

template <typename C> __device__ __forceinline__ const C* twtab(const FftPlan& p);
template <> __device__ __forceinline__ const double2* twtab<double2>(const FftPlan& p) { return p.tw64; }
template <> __device__ __forceinline__ const float2* twtab<float2>(const FftPlan& p) { return p.tw32; }

// Padded shared-memory index: one spare slot every 128 bytes of data.
template <typename C>
__device__ __forceinline__ int pidx(int i) {
  return sizeof(C) == 8 ? i + (i >> 4) : i + (i >> 3);
}
template <typename C>
__host__ __device__ constexpr size_t padded_elems(size_t n) {
  return sizeof(C) == 8 ? n + (n >> 4) + 1 : n + (n >> 3) + 1;
}

// ---------------------------------------------------------------------------
// roots of unity of small order, evaluated by the compiler:
//   exp(-2 pi i k / n) = (root_cos(k, n), -root_sin(k, n))
// k / n is reduced to [0, 1/8] by the symmetries of the circle (exact integer
// comparisons), and cos / sin of the remaining angle x <= pi/4 are the sums of
// their Taylor series, whose terms fall below 1e-20 after 12 steps.
// ---------------------------------------------------------------------------
constexpr double kTwoPi = 6.28318530717958647692528676655900577;

__host__ __device__ constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int i = 1; i < 12; ++i) {
    t *= -x * x / static_cast<double>((2 * i) * (2 * i + 1));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 12; ++i) {
    t *= -x * x / static_cast<double>((2 * i - 1) * (2 * i));
    s += t;
  }
  return s;
}
// cos(2 pi k / n) (want_sin = false) or sin(2 pi k / n) (want_sin = true)
__host__ __device__ constexpr double root_trig(int k, int n, bool want_sin) {
  k %= n;
  if (k < 0) k += n;
  double sign = 1.0;
  if (2 * k > n) {                 // theta > pi: sin(2 pi - theta) = -sin theta
    k = n - k;
    if (want_sin) sign = -sign;
  }
  // now theta = 2 pi k / n in [0, pi]; write theta = pi - phi if theta > pi/2
  if (4 * k > n) {                 // cos(pi - phi) = -cos phi, sin(pi - phi) = sin phi
    k = n - 2 * k;                 // phi = 2 pi k / (2 n)
    n = 2 * n;
    if (!want_sin) sign = -sign;
  }
  // theta = 2 pi k / n in [0, pi/2]; use the complement above pi/4
  if (8 * k > n) {
    const int kc = n - 4 * k;      // pi/2 - theta = 2 pi kc / (4 n)
    const double x = kTwoPi * static_cast<double>(kc) / static_cast<double>(4 * n);
    return sign * (want_sin ? taylor_cos(x) : taylor_sin(x));
  }
  const double x = kTwoPi * static_cast<double>(k) / static_cast<double>(n);
  return sign * (want_sin ? taylor_sin(x) : taylor_cos(x));
}
__host__ __device__ constexpr double root_cos(int k, int n) { return root_trig(k, n, false); }
__host__ __device__ constexpr double root_sin(int k, int n) { return root_trig(k, n, true); }

// ---------------------------------------------------------------------------
// small DFTs X_k = sum_n x_n exp(SIGN 2 pi i n k / R), in registers
// ---------------------------------------------------------------------------
template <int SIGN, typename C>
__device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// y0 = x0 + t1, y1,2 = (x0 - t1/2) +- i s d with t1 = x1 + x2, d = x1 - x2 and
// s = SIGN sqrt(3)/2; the products s d go into the two outputs as fused
// multiply-adds (12 operations per butterfly instead of 14).
template <int SIGN, typename C>
__device__ __forceinline__ void dft3(C* v) {
  using R = decltype(v[0].x);
  const R h = R(0.5);
  const R s = R(SIGN) * R(0.86602540378443864676372317075294);   // SIGN sqrt(3)/2
  const C t1 = v[1] + v[2];
  const C d = v[1] - v[2];
  const C t2 = mk(fma_rn(-h, t1.x, v[0].x), fma_rn(-h, t1.y, v[0].y));
  v[0] = v[0] + t1;
  v[1] = mk(fma_rn(-s, d.y, t2.x), fma_rn(s, d.x, t2.y));
  v[2] = mk(fma_rn(s, d.y, t2.x), fma_rn(-s, d.x, t2.y));
}

template <int SIGN, typename C>
__device__ __forceinline__ void dft4(C* v) {
  C a = v[0] + v[2], b = v[0] - v[2];
  C c = v[1] + v[3], e = rot<SIGN>(v[1] - v[3]);
  v[0] = a + c;
  v[2] = a - c;
  v[1] = b + e;
  v[3] = b - e;
}

template <int SIGN, typename C>
__device__ __forceinline__ void dft5(C* v) {
  using R = decltype(v[0].x);
  const R c1 = R(0.30901699437494742410229341718282);    // cos(2 pi/5)
  const R c2 = R(-0.80901699437494742410229341718282);   // cos(4 pi/5)
  const R s1 = R(0.95105651629515357211643933337938);    // sin(2 pi/5)
  const R s2 = R(0.58778525229247312916870595463907);    // sin(4 pi/5)
  C a1 = v[1] + v[4], b1 = v[1] - v[4];
  C a2 = v[2] + v[3], b2 = v[2] - v[3];
  C r1 = v[0] + c1 * a1 + c2 * a2;
  C r2 = v[0] + c2 * a1 + c1 * a2;
  C i1 = rot<SIGN>(s1 * b1 + s2 * b2);
  C i2 = rot<SIGN>(s2 * b1 - s1 * b2);
  v[0] = v[0] + a1 + a2;
  v[1] = r1 + i1;
  v[4] = r1 - i1;
  v[2] = r2 + i2;
  v[3] = r2 - i2;
}

template <int SIGN, int R, typename C>
__device__ __forceinline__ void dft_small(C* v) {
  if constexpr (R == 2) dft2<SIGN>(v);
  else if constexpr (R == 3) dft3<SIGN>(v);
  else if constexpr (R == 4) dft4<SIGN>(v);
  else if constexpr (R == 5) dft5<SIGN>(v);
}

// ---------------------------------------------------------------------------
// one sub-stage of a register-blocked pass
//   RHO: radix of the stage, SIG: product of the radices before it inside the
//   pass, RG: radix product of the whole pass; v holds the pass's RG entries
//   (entry j at position b L_g + p + j Lp).  ts = M / (Lp SIG RHO).
// ---------------------------------------------------------------------------
template <int SIGN, bool DIT, int RHO, int SIG, int RG, int JP, typename C>
__device__ __forceinline__ void substage_jp(C* v, C wb) {
  using R = decltype(wb.x);
  C t1 = wb;
  if constexpr (JP > 0) {
    constexpr double cr = root_cos(JP, SIG * RHO), sr = -root_sin(JP, SIG * RHO);
    t1 = cmul(wb, mk(R(cr), R(sr)));
  }
  C tq[RHO];
  tq[0] = mk(R(1), R(0));
  if constexpr (RHO > 1) tq[1] = t1;
#pragma unroll
  for (int q = 2; q < RHO; ++q) tq[q] = cmul(tq[q - 1], t1);
#pragma unroll
  for (int jb = 0; jb < RG / (SIG * RHO); ++jb) {
    C e[RHO];
#pragma unroll
    for (int q = 0; q < RHO; ++q) e[q] = v[jb * SIG * RHO + JP + q * SIG];
    if (DIT) {
#pragma unroll
      for (int q = 1; q < RHO; ++q) e[q] = twmul<SIGN>(e[q], tq[q]);
    }
    dft_small<SIGN, RHO>(e);
    if (!DIT) {
#pragma unroll
      for (int q = 1; q < RHO; ++q) e[q] = twmul<SIGN>(e[q], tq[q]);
    }
#pragma unroll
    for (int q = 0; q < RHO; ++q) v[jb * SIG * RHO + JP + q * SIG] = e[q];
  }
  if constexpr (JP + 1 < SIG) substage_jp<SIGN, DIT, RHO, SIG, RG, JP + 1>(v, wb);
}

// One sub-stage of a register-blocked pass.  RHO: radix of the stage, SIG:
// product of the radices before it inside the pass, RG: radix product of the
// whole pass; v holds the pass's RG entries (entry j at position
// b L_g + p + j Lp).  ts = M / (Lp SIG RHO).  The sub-stage's twiddle for
// entry offset jp < SIG is w_{L_s}^p times the compile-time root w_{SIG RHO}^jp.
template <int SIGN, bool DIT, int RHO, int SIG, int RG, typename C>
__device__ __forceinline__ void substage(C* v, int p, int ts, const C* __restrict__ tw) {
  const C wb = __ldg(&tw[p * ts]);   // w_{L_s}^p, L_s = Lp SIG RHO
  substage_jp<SIGN, DIT, RHO, SIG, RG, 0>(v, wb);
}

// A pass of up to three stages (radices RA, RB, RC in DIT order; 1 = absent).
template <int SIGN, bool DIT, int NL, int RA, int RB, int RC, typename C>
__device__ __forceinline__ void run_pass(C* buf, int M, int Lp, const FastDiv& dv,
                                         const C* __restrict__ tw) {
  constexpr int RG = RA * RB * RC;
  const int units = M / RG;
  const int tsA = M / (Lp * RA);
  const int tsB = tsA / RB;
  const int tsC = tsB / RC;
  for (int u = threadIdx.x; u < units * NL; u += blockDim.x) {
    const int line = (NL == 1) ? 0 : u % NL;
    const int unit = (NL == 1) ? u : u / NL;
    const int b = static_cast<int>(fdiv(static_cast<unsigned>(unit), dv));
    const int p = unit - b * Lp;
    const int base = (b * Lp * RG + p) * NL + line;
    const int step = Lp * NL;
    C v[RG];
#pragma unroll
    for (int j = 0; j < RG; ++j) v[j] = buf[pidx<C>(base + j * step)];
    if (DIT) {
      substage<SIGN, DIT, RA, 1, RG>(v, p, tsA, tw);
      if constexpr (RB > 1) substage<SIGN, DIT, RB, RA, RG>(v, p, tsB, tw);
      if constexpr (RC > 1) substage<SIGN, DIT, RC, RA * RB, RG>(v, p, tsC, tw);
    } else {
      if constexpr (RC > 1) substage<SIGN, DIT, RC, RA * RB, RG>(v, p, tsC, tw);
      if constexpr (RB > 1) substage<SIGN, DIT, RB, RA, RG>(v, p, tsB, tw);
      substage<SIGN, DIT, RA, 1, RG>(v, p, tsA, tw);
    }
#pragma unroll
    for (int j = 0; j < RG; ++j) buf[pidx<C>(base + j * step)] = v[j];
  }
}

// One stage of a prime radix R <= kMaxGenericRadix by the O(R^2) definition,
// with the R-th roots of unity taken from the length-M table (R divides M).
template <int SIGN, bool DIT, int NL, typename C>
__device__ void run_generic(C* buf, int M, int R, int Lp, const FastDiv& dv, const C* __restrict__ tw) {
  const int units = M / R;
  const int Lt = Lp * R;
  const int ts = M / Lt;
  const int MR = M / R;
  for (int u = threadIdx.x; u < units * NL; u += blockDim.x) {
    const int line = (NL == 1) ? 0 : u % NL;
    const int unit = (NL == 1) ? u : u / NL;
    const int b = static_cast<int>(fdiv(static_cast<unsigned>(unit), dv));
    const int p = unit - b * Lp;
    const int base = (b * Lt + p) * NL + line;
    const int step = Lp * NL;
    C v[kMaxGenericRadix];
    C o[kMaxGenericRadix];
    for (int q = 0; q < R; ++q) {
      v[q] = buf[pidx<C>(base + q * step)];
      if (DIT && q > 0) v[q] = twmul<SIGN>(v[q], __ldg(&tw[q * p * ts]));
    }
    for (int k = 0; k < R; ++k) {
      C acc = v[0];
      int e = 0;
      for (int n = 1; n < R; ++n) {
        e += k;
        if (e >= R) e -= R;
        acc = acc + twmul<SIGN>(v[n], __ldg(&tw[e * MR]));
      }
      o[k] = acc;
    }
    for (int q = 0; q < R; ++q) {
      C r = o[q];
      if (!DIT && q > 0) r = twmul<SIGN>(r, __ldg(&tw[q * p * ts]));
      buf[pidx<C>(base + q * step)] = r;
    }
  }
}

// Pass metadata copied to shared memory once per kernel (avoids dynamic
// indexing of kernel-parameter arrays).
struct PassSmem {
  int shape[kMaxPasses];
  int R[kMaxPasses];
  int Lp[kMaxPasses];
  FastDiv dv[kMaxPasses];
};

template <typename C>
__device__ __forceinline__ int load_passes(PassSmem& s, const FftPlan& p) {
  constexpr int k = sizeof(C) == 8 ? 1 : 0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < kMaxPasses; ++i) {
      s.shape[i] = p.pshape[k][i];
      s.R[i] = p.pR[k][i];
      s.Lp[i] = p.pLp[k][i];
      s.dv[i] = p.pdiv[k][i];
    }
  }
  return p.npass[k];
}

// Passes wider than 18 entries run only in FP32 (the FP64 plans never use them,
// and leaving them out keeps the FP64 kernels' register allocation small).
template <int SIGN, bool DIT, int NL, int RA, int RB, int RC, typename C>
__device__ __forceinline__ void run_pass_p(C* buf, int M, int Lp, const FastDiv& dv,
                                           const C* __restrict__ tw) {
  if constexpr (sizeof(C) == 8 || RA * RB * RC <= 18) run_pass<SIGN, DIT, NL, RA, RB, RC>(buf, M, Lp, dv, tw);
}

template <int SIGN, bool DIT, int NL, typename C>
__device__ __forceinline__ void dispatch_pass(C* buf, int M, const PassSmem& ps, int i,
                                              const C* __restrict__ tw) {
  const int Lp = ps.Lp[i];
  const FastDiv dv = ps.dv[i];
  switch (ps.shape[i]) {
    case SH_2: run_pass_p<SIGN, DIT, NL, 2, 1, 1>(buf, M, Lp, dv, tw); break;
    case SH_3: run_pass_p<SIGN, DIT, NL, 3, 1, 1>(buf, M, Lp, dv, tw); break;
    case SH_4: run_pass_p<SIGN, DIT, NL, 4, 1, 1>(buf, M, Lp, dv, tw); break;
    case SH_5: run_pass_p<SIGN, DIT, NL, 5, 1, 1>(buf, M, Lp, dv, tw); break;
    case SH_2_3: run_pass_p<SIGN, DIT, NL, 2, 3, 1>(buf, M, Lp, dv, tw); break;
    case SH_3_3: run_pass_p<SIGN, DIT, NL, 3, 3, 1>(buf, M, Lp, dv, tw); break;
    case SH_2_5: run_pass_p<SIGN, DIT, NL, 2, 5, 1>(buf, M, Lp, dv, tw); break;
    case SH_4_3: run_pass_p<SIGN, DIT, NL, 4, 3, 1>(buf, M, Lp, dv, tw); break;
    case SH_3_5: run_pass_p<SIGN, DIT, NL, 3, 5, 1>(buf, M, Lp, dv, tw); break;
    case SH_4_4: run_pass_p<SIGN, DIT, NL, 4, 4, 1>(buf, M, Lp, dv, tw); break;
    case SH_4_5: run_pass_p<SIGN, DIT, NL, 4, 5, 1>(buf, M, Lp, dv, tw); break;
    case SH_5_5: run_pass_p<SIGN, DIT, NL, 5, 5, 1>(buf, M, Lp, dv, tw); break;
    case SH_4_2: run_pass_p<SIGN, DIT, NL, 4, 2, 1>(buf, M, Lp, dv, tw); break;
    case SH_2_3_3: run_pass_p<SIGN, DIT, NL, 2, 3, 3>(buf, M, Lp, dv, tw); break;
    case SH_3_3_3: run_pass_p<SIGN, DIT, NL, 3, 3, 3>(buf, M, Lp, dv, tw); break;
    case SH_4_2_3: run_pass_p<SIGN, DIT, NL, 4, 2, 3>(buf, M, Lp, dv, tw); break;
    case SH_2_3_5: run_pass_p<SIGN, DIT, NL, 2, 3, 5>(buf, M, Lp, dv, tw); break;
    case SH_4_4_2: run_pass_p<SIGN, DIT, NL, 4, 4, 2>(buf, M, Lp, dv, tw); break;
    default: run_generic<SIGN, DIT, NL>(buf, M, ps.R[i], Lp, dv, tw); break;
  }
}

// Decimation in time: digit-reversed input -> natural output.  The caller
// must __syncthreads() after filling buf; returns after a final barrier.
template <int SIGN, int NL, typename C>
__device__ void fft_dit(C* buf, const PassSmem& ps, int npass, int M, const C* tw) {
  for (int i = 0; i < npass; ++i) {
    dispatch_pass<SIGN, true, NL>(buf, M, ps, i, tw);
    __syncthreads();
  }
}

// Decimation in frequency: natural input -> digit-reversed output.
template <int SIGN, int NL, typename C>
__device__ void fft_dif(C* buf, const PassSmem& ps, int npass, int M, const C* tw) {
  for (int i = npass - 1; i >= 0; --i) {
    dispatch_pass<SIGN, false, NL>(buf, M, ps, i, tw);
    __syncthreads();
  }
}

}  // namespace ghb
