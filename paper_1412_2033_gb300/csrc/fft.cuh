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
// buf[m * NL + line], so that consecutive threads touch consecutive words.
//
// Algorithms (in place, one shared buffer, one barrier per stage):
//  * fft_dit: decimation in time.  Input in mixed-radix digit-reversed order
//    (the caller scatters x[n] to position perm[n]), output in natural order.
//    Stage t (radix R_t, L_{t-1} = R_1...R_{t-1}, L_t = L_{t-1} R_t) combines
//    R_t transforms of length L_{t-1}: for block b and position p < L_{t-1} the
//    butterfly reads the R_t entries b L_t + p + q L_{t-1}, multiplies entry q by
//    w_{L_t}^{pq}, applies DFT_{R_t} and writes back in place.
//  * fft_dif: decimation in frequency, the same stages in reverse order with
//    the twiddle applied after the small DFT.  Input natural, output
//    digit-reversed (X[k] ends at position perm[k]).
// The pair lets a line go inverse (DIT) -> pointwise multiply in natural order
// -> forward (DIF) without any permutation pass.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace ghb {

constexpr int kMaxStages = 24;
constexpr int kMaxGenericRadix = 31;

// Plan of one length-M transform.  Tables live in device memory.
struct FftPlan {
  int M;
  int nst;                   // number of stages
  int R[kMaxStages];         // radix of DIT stage t
  int Lp[kMaxStages];        // L_{t-1}: product of the radices before stage t
  const int* perm;           // perm[n]: digit-reversed position of index n
  const double2* tw64;       // tw64[j] = exp(-2 pi i j / M)
  const float2* tw32;        // the same rounded to float
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

// a * w (SIGN = -1) or a * conj(w) (SIGN = +1); w from the forward table.
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

// Small DFTs X_k = sum_n x_n exp(SIGN 2 pi i n k / R), in registers.
template <int SIGN, typename C>
__device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <int SIGN, typename C>
__device__ __forceinline__ void dft3(C* v) {
  using R = decltype(v[0].x);
  const R h = R(0.5);
  const R s3 = R(0.86602540378443864676372317075294);   // sqrt(3)/2
  C t1 = v[1] + v[2];
  C t2 = v[0] - h * t1;
  C t3 = s3 * rot<SIGN>(v[1] - v[2]);
  v[0] = v[0] + t1;
  v[1] = t2 + t3;
  v[2] = t2 - t3;
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
  if (R == 2) dft2<SIGN>(v);
  else if (R == 3) dft3<SIGN>(v);
  else if (R == 4) dft4<SIGN>(v);
  else if (R == 5) dft5<SIGN>(v);
}

// Butterfly of a specialised radix.  DIT: twiddle, then DFT; DIF: DFT, then twiddle.
template <int SIGN, int R, bool DIT, typename C>
__device__ __forceinline__ void bfly(C* buf, int base, int step, int twj, const C* tw) {
  C v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = buf[base + q * step];
  if (DIT) {
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = twmul<SIGN>(v[q], __ldg(&tw[q * twj]));
  }
  dft_small<SIGN, R>(v);
  if (!DIT) {
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = twmul<SIGN>(v[q], __ldg(&tw[q * twj]));
  }
#pragma unroll
  for (int q = 0; q < R; ++q) buf[base + q * step] = v[q];
}

// Butterfly of any radix R <= kMaxGenericRadix by the O(R^2) definition, with
// the R-th roots of unity taken from the length-M table (R divides M).
template <int SIGN, bool DIT, typename C>
__device__ void bfly_generic(C* buf, int base, int step, int twj, int R, int M, const C* tw) {
  C v[kMaxGenericRadix];
  C o[kMaxGenericRadix];
  const int MR = M / R;
  for (int q = 0; q < R; ++q) {
    v[q] = buf[base + q * step];
    if (DIT && q > 0) v[q] = twmul<SIGN>(v[q], __ldg(&tw[q * twj]));
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
    if (!DIT && q > 0) r = twmul<SIGN>(r, __ldg(&tw[q * twj]));
    buf[base + q * step] = r;
  }
}

// Stage metadata copied to shared memory once per kernel (avoids dynamic
// indexing of kernel-parameter arrays).
struct StageSmem {
  int R[kMaxStages];
  int Lp[kMaxStages];
};

__device__ __forceinline__ void load_stages(StageSmem& s, const FftPlan& p) {
#pragma unroll
  for (int i = 0; i < kMaxStages; ++i) {
    if (threadIdx.x == 0) {
      s.R[i] = p.R[i];
      s.Lp[i] = p.Lp[i];
    }
  }
}

// One stage over NL interleaved lines.
template <int SIGN, bool DIT, int NL, typename C>
__device__ __forceinline__ void fft_stage(C* buf, int M, int R, int Lp, const C* tw) {
  const int Lt = Lp * R;
  const int nb = M / R;
  const int tws = M / Lt;
  const int total = nb * NL;
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    const int line = (NL == 1) ? 0 : (u % NL);
    const int beta = (NL == 1) ? u : (u / NL);
    const int b = beta / Lp;
    const int p = beta - b * Lp;
    const int base = (b * Lt + p) * NL + line;
    const int step = Lp * NL;
    const int twj = p * tws;
    switch (R) {
      case 2: bfly<SIGN, 2, DIT>(buf, base, step, twj, tw); break;
      case 3: bfly<SIGN, 3, DIT>(buf, base, step, twj, tw); break;
      case 4: bfly<SIGN, 4, DIT>(buf, base, step, twj, tw); break;
      case 5: bfly<SIGN, 5, DIT>(buf, base, step, twj, tw); break;
      default: bfly_generic<SIGN, DIT>(buf, base, step, twj, R, M, tw); break;
    }
  }
}

// Decimation in time: digit-reversed input -> natural output.  The caller
// must __syncthreads() after filling buf; returns after a final barrier.
template <int SIGN, int NL, typename C>
__device__ void fft_dit(C* buf, const StageSmem& st, int nst, int M, const C* tw) {
  for (int s = 0; s < nst; ++s) {
    fft_stage<SIGN, true, NL>(buf, M, st.R[s], st.Lp[s], tw);
    __syncthreads();
  }
}

// Decimation in frequency: natural input -> digit-reversed output.
template <int SIGN, int NL, typename C>
__device__ void fft_dif(C* buf, const StageSmem& st, int nst, int M, const C* tw) {
  for (int s = nst - 1; s >= 0; --s) {
    fft_stage<SIGN, false, NL>(buf, M, st.R[s], st.Lp[s], tw);
    __syncthreads();
  }
}

}  // namespace ghb
