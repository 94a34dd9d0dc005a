// Field-level kernels: coefficient tables, right-hand sides, projections and
// the conjugate-gradient vector updates with their FP64 reductions.
//
// Fields are half spectra on Z_N (see ghb.h): x[c][i_1]..[i_{d-1}][j].  The
// inner product of the paper's complex space (Section 5.1,
// (u, v) = sum_{k in Z_N} u(k).conj v(k)) is evaluated on the half spectrum as
// sum_k w_k Re(u(k).conj v(k)) with weight w_k = 1 on the plane k_d = 0 and 2
// elsewhere (each stored k_d > 0 stands for k and -k).
#include <algorithm>
#include <atomic>
#include <cmath>

#include "ghb_internal.cuh"
#include "reduce.cuh"

namespace ghb {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kFieldThreads = 256;

int field_grid(int64_t n) {
  int64_t b = (n + kFieldThreads - 1) / kFieldThreads;
  if (b > 1216) b = 1216;   // 152 SMs x 8
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

__device__ __forceinline__ void kvec(const FieldGeom& g, int64_t e64, int k[3], int& j) {
  // 32-bit index arithmetic: a field has fewer than 2^31 entries per component
  const unsigned e = static_cast<unsigned>(e64);
  const unsigned h = static_cast<unsigned>(g.h);
  const unsigned i12 = fdiv(e, g.hdiv);
  j = static_cast<int>(e - i12 * h);
  if (g.d == 2) {
    k[0] = static_cast<int>(i12) - (g.N[0] - 1) / 2;
    k[1] = j;
    k[2] = 0;
  } else {
    const unsigned n1 = static_cast<unsigned>(g.N[1]);
    const unsigned i1 = fdiv(i12, g.n1div);
    const unsigned i2 = i12 - i1 * n1;
    k[0] = static_cast<int>(i1) - (g.N[0] - 1) / 2;
    k[1] = static_cast<int>(i2) - (g.N[1] - 1) / 2;
    k[2] = j;
  }
}

// Last-axis frequency j of entry e (e mod h).
__device__ __forceinline__ int jindex(const FieldGeom& g, int64_t e64) {
  const unsigned e = static_cast<unsigned>(e64);
  return static_cast<int>(e - fdiv(e, g.hdiv) * static_cast<unsigned>(g.h));
}

// Index of the entry holding -k for an entry on the plane k_d = 0 (where both
// k and -k are stored); -1 elsewhere.
__device__ __forceinline__ int64_t mirror_index(const FieldGeom& g, const int k[3], int j) {
  if (j != 0) return -1;
  const int i1 = (g.N[0] - 1) / 2 - k[0];
  if (g.d == 2) return static_cast<int64_t>(i1) * g.h;
  const int i2 = (g.N[1] - 1) / 2 - k[1];
  return (static_cast<int64_t>(i1) * g.N[1] + i2) * g.h;
}

// Real part of a field on Z_N (Def. trig_pol: admissible fields are real
// trigonometric polynomials, w(-k) = conj w(k)).  Only the plane k_d = 0 holds
// both k and -k; there the Hermitian part (w(k) + conj w(-k))/2 is taken.
template <typename C>
__device__ __forceinline__ C hermitian_part(const C* w, int64_t P, int c, int64_t e, int64_t em) {
  const C a = w[c * P + e];
  if (em < 0) return a;
  const C b = w[c * P + em];
  using T = decltype(a.x);
  return mk(T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y));
}

// q = G(k) w with G_E = k k^T / k.k (primal) or G_J = I - G_E (dual), 0 at k = 0
// (Def. projection).
template <typename T, typename C>
__device__ __forceinline__ void project_vec(int d, const int k[3], int kind, const C* w, C* q) {
  const T k0 = T(k[0]), k1 = T(k[1]), k2 = T(k[2]);
  const T kk = k0 * k0 + k1 * k1 + k2 * k2;
  if (kk == T(0)) {
    for (int c = 0; c < d; ++c) q[c] = mk(T(0), T(0));
    return;
  }
  const T kv[3] = {k0, k1, k2};
  T sx = T(0), sy = T(0);
  for (int c = 0; c < d; ++c) {
    sx += kv[c] * w[c].x;
    sy += kv[c] * w[c].y;
  }
  const T inv = T(1) / kk;   // one division per entry
  sx *= inv;
  sy *= inv;
  for (int c = 0; c < d; ++c) {
    const C pe = mk(kv[c] * sx, kv[c] * sy);
    q[c] = (kind == GHB_PRIMAL) ? pe : mk(w[c].x - pe.x, w[c].y - pe.y);
  }
}

// Grid-wide sum: partial per block, the last block to finish adds the
// partials in block order.  Returns true in thread 0 of that block with *total.
// `bid`, `nb`: this block and the number of blocks working on the same operand.
__device__ bool grid_sum_last(double v, double* partials, unsigned int* ticket, double* total,
                              int64_t bid, int64_t nb) {
  __shared__ double red[32];
  __shared__ bool last;
  const double bs = block_sum(v, red);
  if (threadIdx.x == 0) {
    partials[bid] = bs;
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(&partials[b]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    *total = s;
    return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// coefficient table (eq. inclcomp_formula with the shape coefficients of
// Remark anal_Fourier; the sphere by its radial transform)
// ---------------------------------------------------------------------------
__device__ double sinc_pi(double x) {   // sin(pi x)/(pi x)
  return x == 0.0 ? 1.0 : sinpi(x) / (kPi * x);
}

// Bessel function of the first kind of order one.
//  |x| <= 8: CUDA's j1 (accurate to a few ulp there).
//  8 < |x| < 20: Miller's backward recurrence J_{n-1} = (2n/x) J_n - J_{n+1},
//     started at n0 ~ |x| + 40 with J_{n0+1} = 0, normalised by the identity
//     J_0 + 2 sum_{k>=1} J_{2k} = 1.
//  |x| >= 20: Hankel's asymptotic expansion (Abramowitz and Stegun 9.2.5,
//     9.2.9-9.2.10): J_1(x) = sqrt(2/(pi x)) (P cos chi - Q sin chi),
//     chi = x - 3 pi/4, P = sum_k (-1)^k a_{2k} x^{-2k},
//     Q = sum_k (-1)^k a_{2k+1} x^{-2k-1},
//     a_m = prod_{j=1..m} (4 - (2j-1)^2) / (m! 8^m); summed until the terms
//     fall below 1e-18 (the smallest term is about e^{-2x}).
// CUDA's j1 loses about 1e-12 relative to the envelope sqrt(2/(pi x)) beyond
// x = 8, which is visible in the bounds at the 1e-13 level.
__device__ double bessel_j1(double x) {
  const double ax = fabs(x);
  const double sg = x < 0 ? -1.0 : 1.0;
  if (ax <= 8.0) return j1(x);
  if (ax < 20.0) {
    int n0 = static_cast<int>(ax) + 40;
    n0 += n0 & 1;                       // even start
    double jp1 = 0.0, jn = 1e-30, sum = 2.0 * jn, j1v = 0.0;
    for (int n = n0; n >= 1; --n) {
      const double jm1 = (2.0 * n / ax) * jn - jp1;   // J_{n-1}
      jp1 = jn;
      jn = jm1;
      const int m = n - 1;
      if (m == 1) j1v = jn;
      if ((m & 1) == 0) sum += (m == 0 ? 1.0 : 2.0) * jn;
      if (fabs(jn) > 1e200) {          // rescale to stay in range
        jn *= 1e-200;
        jp1 *= 1e-200;
        sum *= 1e-200;
        j1v *= 1e-200;
      }
    }
    return sg * j1v / sum;
  }
  const double inv = 1.0 / ax;
  double P = 1.0, Q = 0.0;
  double a = 1.0;                        // a_m x^{-m} with alternating signs folded in below
  for (int m = 1; m < 60; ++m) {
    a *= (4.0 - (2.0 * m - 1.0) * (2.0 * m - 1.0)) / (8.0 * m) * inv;
    // m odd -> Q term (-1)^((m-1)/2), m even -> P term (-1)^(m/2)
    const int k = m >> 1;
    const double term = ((k & 1) ? -a : a);
    if (m & 1) Q += term;
    else P += term;
    if (fabs(a) < 1e-18) break;
  }
  double s, c;
  sincos(ax, &s, &c);
  const double r2 = 0.70710678118654752440084436210485;   // 1/sqrt(2)
  const double cchi = (s - c) * r2;       // cos(x - 3 pi / 4)
  const double schi = -(s + c) * r2;      // sin(x - 3 pi / 4)
  return sg * sqrt(2.0 / (kPi * ax)) * (P * cchi - Q * schi);
}

__device__ double shape_coeff(const Incl& in, int d, const int n[3]) {
  if (in.shape == GHB_BOX) {
    double v = 1.0;
    for (int a = 0; a < d; ++a) v *= in.s[a] * sinc_pi(in.s[a] * n[a]);
    return v;
  }
  const double r = in.s[0];
  const double rho2 = double(n[0]) * n[0] + double(n[1]) * n[1] + double(n[2]) * n[2];
  const double rho = sqrt(rho2);
  if (in.shape == GHB_DISK) {
    if (rho2 == 0.0) return kPi * r * r;
    return r * bessel_j1(2.0 * kPi * r * rho) / rho;
  }
  // sphere
  const double q = 2.0 * kPi * r * rho;
  if (q < 1e-2) {
    const double q2 = q * q;
    return 4.0 / 3.0 * kPi * r * r * r * (1.0 - q2 / 10.0 + q2 * q2 / 280.0 - q2 * q2 * q2 / 15120.0);
  }
  double sq, cq;
  sincos(q, &sq, &cq);
  return (sq - q * cq) / (2.0 * kPi * kPi * rho2 * rho);
}

// tab1 (optional): the table of a second inclusion list with the same shapes
// and centres (the coefficient 1/a beside a); each inclusion's shape factor and
// phase are evaluated once for both.  Every shape factor is even in each
// component of n (products of sinc for boxes, functions of |n| for disks and
// spheres), so one thread takes n = (n_0, ...) with n_0 >= 0 together with
// its mirror (-n_0, ...): each shape factor once, the phase of each entry as
// before (the same operations per entry, so the same values).
__global__ void coeff_kernel(double2* tab, double2* tab1, Geometry g, const Incl* incs, const Incl* incs1, int n,
                             double a0v, double a0v1) {
  const int d = g.d;
  const int N0 = g.N[0];
  const int L1 = (d == 3) ? 2 * g.N[1] - 1 : g.N[1];
  const int Ld = g.N[d - 1];   // half of 2N_d - 1: n_d = 0..N_d-1
  const int64_t rest = (d == 3) ? static_cast<int64_t>(L1) * Ld : Ld;   // entries per value of n_0
  const int64_t half = static_cast<int64_t>(N0) * rest;                 // n_0 = 0 .. N_0-1
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < half;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t n0 = e / rest;
    const int64_t rr = e - n0 * rest;
    int nv[3] = {static_cast<int>(n0), 0, 0};
    if (d == 2) {
      nv[1] = static_cast<int>(rr);
    } else {
      const int64_t i1 = rr / Ld;
      nv[1] = static_cast<int>(i1) - (g.N[1] - 1);
      nv[2] = static_cast<int>(rr - i1 * Ld);
    }
    const int nm[3] = {-nv[0], nv[1], nv[2]};
    const bool mirror = nv[0] != 0;
    const bool origin = nv[0] == 0 && nv[1] == 0 && nv[2] == 0;
    double re = origin ? a0v : 0.0, im = 0.0;
    double re1 = origin ? a0v1 : 0.0, im1 = 0.0;
    double rem = 0.0, imm = 0.0, rem1 = 0.0, imm1 = 0.0;   // the mirror entry
    for (int i = 0; i < n; ++i) {
      const Incl in = incs[i];
      const double sh = shape_coeff(in, d, nv);
      const double f = in.dv * sh;
      const double f1 = tab1 != nullptr ? incs1[i].dv * sh : 0.0;
      // exp(-2 pi i n.x_i): reduce n.x_i to [-1/2, 1/2] before the sincos
      double t = 0.0;
      for (int a = 0; a < d; ++a) t = fma(static_cast<double>(nv[a]), in.c[a], t);
      t -= rint(t);
      double s, c;
      sincospi(2.0 * t, &s, &c);
      re += f * c;
      im -= f * s;
      re1 += f1 * c;
      im1 -= f1 * s;
      if (mirror) {
        double tm = 0.0;
        for (int a = 0; a < d; ++a) tm = fma(static_cast<double>(nm[a]), in.c[a], tm);
        tm -= rint(tm);
        sincospi(2.0 * tm, &s, &c);
        rem += f * c;
        imm -= f * s;
        rem1 += f1 * c;
        imm1 -= f1 * s;
      }
    }
    const int64_t ep = (n0 + N0 - 1) * rest + rr, em = (N0 - 1 - n0) * rest + rr;
    tab[ep] = make_double2(re, im);
    if (tab1 != nullptr) tab1[ep] = make_double2(re1, im1);
    if (mirror) {
      tab[em] = make_double2(rem, imm);
      if (tab1 != nullptr) tab1[em] = make_double2(rem1, imm1);
    }
  }
}

// ---------------------------------------------------------------------------
// right-hand side b(k) = -G(k) a^(k) E (Prop. min2linear_sys; (A^full E^)(k) = a^(k) E)
// ---------------------------------------------------------------------------
__global__ void rhs_kernel(double2* b, const double2* tab, Geometry g, FieldGeom fg, double3 E,
                           int kind) {
  const int d = fg.d;
  const int Ld = g.N[d - 1];
  const int L1 = 2 * g.N[1] - 1;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int k[3];
    int j;
    kvec(fg, e, k, j);
    int64_t ti;
    if (d == 2) ti = static_cast<int64_t>(k[0] + g.N[0] - 1) * Ld + j;
    else ti = (static_cast<int64_t>(k[0] + g.N[0] - 1) * L1 + (k[1] + g.N[1] - 1)) * Ld + j;
    const double2 a = tab[ti];
    const double Ev[3] = {E.x, E.y, E.z};
    double2 w[3], q[3];
    for (int c = 0; c < d; ++c) w[c] = make_double2(a.x * Ev[c], a.y * Ev[c]);
    project_vec<double>(d, k, kind, w, q);
    for (int c = 0; c < d; ++c) b[c * fg.P + e] = make_double2(-q[c].x, -q[c].y);
  }
}

// ---------------------------------------------------------------------------
// CG vector operations on one operand (CgItem), executed by blocks
// bid = 0..nb-1; used by one-operand launches and by batched launches over
// many operands alike.
// ---------------------------------------------------------------------------
#define GHB_FIELD_LOOP(e, fg, bid, nb)                                                  \
  for (int64_t e = (bid) * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < (fg).P; \
       e += (nb) * static_cast<int64_t>(blockDim.x))

// The per-entry loops below take the dimension as a template parameter D so
// that the component arrays stay in registers.

// q = G w (with the Hermitian part taken on k_d = 0); q must not alias w.
template <typename T, int D>
__device__ __forceinline__ void project_loop(const CgItem& it, int64_t bid, int64_t nb) {
  using C = typename CT<T>::type;
  const FieldGeom& fg = it.fg;
  const C* w = static_cast<const C*>(it.w);
  C* y = static_cast<C*>(it.q);
  GHB_FIELD_LOOP(e, fg, bid, nb) {
    int k[3];
    int j;
    kvec(fg, e, k, j);
    const int64_t em = mirror_index(fg, k, j);
    C wv[D], q[D];
#pragma unroll
    for (int c = 0; c < D; ++c) wv[c] = hermitian_part(w, fg.P, c, e, em);
    project_vec<T>(D, k, it.kind, wv, q);
#pragma unroll
    for (int c = 0; c < D; ++c) y[c * fg.P + e] = q[c];
  }
}
template <typename T>
__device__ void op_project(const CgItem& it, int64_t bid, int64_t nb) {
  if (it.fg.d == 2) project_loop<T, 2>(it, bid, nb);
  else project_loop<T, 3>(it, bid, nb);
}

// x = 0, r = b, p = 0, <b, b>; the last block initialises the CG scalars.
template <typename T>
__device__ void op_init(const CgItem& it, int64_t bid, int64_t nb) {
  using C = typename CT<T>::type;
  const FieldGeom& fg = it.fg;
  C* x = static_cast<C*>(it.x);
  C* r = static_cast<C*>(it.r);
  C* p = static_cast<C*>(it.p);
  const C* b = static_cast<const C*>(it.b);
  CgState* st = it.st;
  // per-thread partial sums in the field's precision (a few dozen terms), the
  // cross-thread and cross-block sums in FP64
  T acc = T(0);
  GHB_FIELD_LOOP(e, fg, bid, nb) {
    const int j = jindex(fg, e);
    const T wt = (j == 0) ? T(1) : T(2);
    for (int c = 0; c < fg.d; ++c) {
      const int64_t i = c * fg.P + e;
      const C bv = b[i];
      x[i] = mk(T(0), T(0));
      p[i] = mk(T(0), T(0));
      r[i] = bv;
      acc += wt * (bv.x * bv.x + bv.y * bv.y);
    }
  }
  double tot;
  if (grid_sum_last(static_cast<double>(acc), it.partials, &st->ticket, &tot, bid, nb)) {
    st->bb = tot;
    st->rr = tot;
    st->tol2 = it.tol * it.tol * tot;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->pq = 0.0;
    st->iter = 0;
    st->maxiter = it.maxiter;
    st->done = (tot == 0.0) ? CONVERGED : RUNNING;
    st->dec = 0.0;
    if (st->hist != nullptr && st->hist_cap > 0) st->hist[0] = 0.0;
  }
}

// Per-thread part of op_project_dot: q = G w on this thread's entries and
// their share of <p, q> (in the field's precision).
template <typename T, int D>
__device__ __forceinline__ T project_dot_loop(const CgItem& it, int64_t bid, int64_t nb) {
  using C = typename CT<T>::type;
  const FieldGeom& fg = it.fg;
  C* q = static_cast<C*>(it.q);
  const C* w = static_cast<const C*>(it.w);
  const C* p = static_cast<const C*>(it.p);
  T acc = T(0);
  GHB_FIELD_LOOP(e, fg, bid, nb) {
    int k[3];
    int j;
    kvec(fg, e, k, j);
    const T wt = (j == 0) ? T(1) : T(2);
    const int64_t em = mirror_index(fg, k, j);
    C wv[D], pv[D], qv[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      wv[c] = hermitian_part(w, fg.P, c, e, em);
      pv[c] = p[c * fg.P + e];
    }
    project_vec<T>(D, k, it.kind, wv, qv);
    T sacc = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      q[c * fg.P + e] = qv[c];
      sacc += pv[c].x * qv[c].x + pv[c].y * qv[c].y;
    }
    acc += wt * sacc;
  }
  return acc;
}

// q = G w, <p, q>; the last block forms alpha = <r, r> / <p, A p>.
template <typename T>
__device__ void op_project_dot(const CgItem& it, int64_t bid, int64_t nb) {
  const FieldGeom& fg = it.fg;
  CgState* st = it.st;
  if (st->done != RUNNING) return;
  const T acc = fg.d == 2 ? project_dot_loop<T, 2>(it, bid, nb) : project_dot_loop<T, 3>(it, bid, nb);
  double tot;
  if (grid_sum_last(static_cast<double>(acc), it.partials, &st->ticket, &tot, bid, nb)) {
    st->pq = tot;
    if (!(tot > 0.0) || !isfinite(tot)) {
      st->done = BREAKDOWN;
      st->alpha = 0.0;
    } else {
      st->alpha = st->rr / tot;
    }
  }
}

// Per-thread part of op_update: x += alpha p, r -= alpha q on this thread's
// entries and their share of <r, r>.
template <typename T, int D>
__device__ __forceinline__ T update_loop(const CgItem& it, T al, int64_t bid, int64_t nb) {
  using C = typename CT<T>::type;
  const FieldGeom& fg = it.fg;
  C* x = static_cast<C*>(it.x);
  C* r = static_cast<C*>(it.r);
  const C* p = static_cast<const C*>(it.p);
  const C* q = static_cast<const C*>(it.q);
  T acc = T(0);
  GHB_FIELD_LOOP(e, fg, bid, nb) {
    const int j = jindex(fg, e);
    const T wt = (j == 0) ? T(1) : T(2);
    C pv[D], qv[D], xv[D], rv[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const int64_t i = c * fg.P + e;
      pv[c] = p[i];
      qv[c] = q[i];
      xv[c] = x[i];
      rv[c] = r[i];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const int64_t i = c * fg.P + e;
      const C xn = mk(xv[c].x + al * pv[c].x, xv[c].y + al * pv[c].y);
      const C rn = mk(rv[c].x - al * qv[c].x, rv[c].y - al * qv[c].y);
      x[i] = xn;
      r[i] = rn;
      acc += wt * (rn.x * rn.x + rn.y * rn.y);
    }
  }
  return acc;
}

// x += alpha p, r -= alpha q, <r, r>; the last block forms beta and the stop test.
template <typename T>
__device__ void op_update(const CgItem& it, int64_t bid, int64_t nb) {
  const FieldGeom& fg = it.fg;
  CgState* st = it.st;
  if (st->done != RUNNING) return;
  const T al = static_cast<T>(st->alpha);
  // per-thread partial in the field's precision, FP64 across threads
  const T acc = fg.d == 2 ? update_loop<T, 2>(it, al, bid, nb) : update_loop<T, 3>(it, al, bid, nb);
  double tot;
  if (grid_sum_last(static_cast<double>(acc), it.partials, &st->ticket, &tot, bid, nb)) {
    const double rr_old = st->rr;
    st->beta = tot / rr_old;
    st->rr = tot;
    st->dec += st->alpha * rr_old;
    st->iter += 1;
    if (st->hist != nullptr && st->iter < st->hist_cap) st->hist[st->iter] = st->dec;
    if (!isfinite(tot)) st->done = BREAKDOWN;
    else if (tot <= st->tol2) st->done = CONVERGED;
    else if (st->iter >= st->maxiter) st->done = MAXITER;
  }
}

// FP64 residual r = b - w and <r, r> into st->rr.
__device__ void op_residual(const CgItem& it, int64_t bid, int64_t nb) {
  const FieldGeom& fg = it.fg;
  double2* r = static_cast<double2*>(it.r);
  const double2* b = static_cast<const double2*>(it.b);
  const double2* y = static_cast<const double2*>(it.w);
  double acc = 0.0;
  GHB_FIELD_LOOP(e, fg, bid, nb) {
    const int j = jindex(fg, e);
    const double wt = (j == 0) ? 1.0 : 2.0;
    for (int c = 0; c < fg.d; ++c) {
      const int64_t i = c * fg.P + e;
      const double2 rv = make_double2(b[i].x - y[i].x, b[i].y - y[i].y);
      r[i] = rv;
      acc += wt * (rv.x * rv.x + rv.y * rv.y);
    }
  }
  double tot;
  if (grid_sum_last(acc, it.partials, &it.st->ticket, &tot, bid, nb)) it.st->rr = tot;
}

// FP32 copy q = (float) w of an FP64 field.
__device__ void op_to_f32(const CgItem& it, int64_t bid, int64_t nb) {
  const FieldGeom& fg = it.fg;
  float2* dst = static_cast<float2*>(it.q);
  const double2* src = static_cast<const double2*>(it.w);
  GHB_FIELD_LOOP(e, fg, bid, nb) {
    for (int c = 0; c < fg.d; ++c) {
      const int64_t i = c * fg.P + e;
      dst[i] = make_float2(static_cast<float>(src[i].x), static_cast<float>(src[i].y));
    }
  }
}

// FP64 accumulation x = w + (double) p with p an FP32 correction.
__device__ void op_accum(const CgItem& it, int64_t bid, int64_t nb) {
  const FieldGeom& fg = it.fg;
  double2* x = static_cast<double2*>(it.x);
  const double2* w = static_cast<const double2*>(it.w);
  const float2* dx = static_cast<const float2*>(it.p);
  GHB_FIELD_LOOP(e, fg, bid, nb) {
    for (int c = 0; c < fg.d; ++c) {
      const int64_t i = c * fg.P + e;
      x[i] = make_double2(w[i].x + static_cast<double>(dx[i].x), w[i].y + static_cast<double>(dx[i].y));
    }
  }
}

template <typename T, int OP>
__device__ __forceinline__ void run_op(const CgItem& it, int64_t bid, int64_t nb) {
  if constexpr (OP == CG_INIT) op_init<T>(it, bid, nb);
  else if constexpr (OP == CG_PROJECT_DOT) op_project_dot<T>(it, bid, nb);
  else if constexpr (OP == CG_UPDATE) op_update<T>(it, bid, nb);
  else if constexpr (OP == CG_PROJECT) op_project<T>(it, bid, nb);
  else if constexpr (OP == CG_RESIDUAL) op_residual(it, bid, nb);
  else if constexpr (OP == CG_TO_F32) op_to_f32(it, bid, nb);
  else if constexpr (OP == CG_ACCUM) op_accum(it, bid, nb);
}

template <typename T, int OP>
__global__ void __launch_bounds__(kFieldThreads) cg_kernel(CgItem it) {
  run_op<T, OP>(it, blockIdx.x, gridDim.x);
}

template <typename Item>
__device__ __forceinline__ int find_cg_item(const Item* items, int n, int64_t b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].block_begin <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, int OP>
__global__ void __launch_bounds__(kFieldThreads) cg_kernel_batch(const CgItem* __restrict__ items, int n) {
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = find_cg_item(items, n, blockIdx.x);
  __syncthreads();
  const CgItem& it = items[s_item];
  run_op<T, OP>(it, blockIdx.x - it.block_begin, it.nblocks);
}

__global__ void to_f32_real_kernel(float* dst, const double* src, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[i] = static_cast<float>(src[i]);
}

__global__ void add_constant_kernel(double2* v, const double2* e, FieldGeom fg, double3 E,
                                    int64_t e0) {
  const double Ev[3] = {E.x, E.y, E.z};
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < fg.P;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int c = 0; c < fg.d; ++c) {
      double2 val = e[c * fg.P + i];
      if (i == e0) val.x += Ev[c];
      v[c * fg.P + i] = val;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
ghb_status launch_coeff_tables(double2* tab0, double2* tab1, const Geometry& g, const Incl* incs0,
                               const Incl* incs1, int n, double a0v0, double a0v1, cudaStream_t s) {
  const int64_t half = static_cast<int64_t>(g.N[0]) * (g.table / (2 * g.N[0] - 1));   // n_0 >= 0
  coeff_kernel<<<field_grid(half), kFieldThreads, 0, s>>>(tab0, tab1, g, incs0, incs1, n, a0v0, a0v1);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

template <typename T>
ghb_status launch_rhs(void* b, const double2* tab, const Geometry& g, const double* E, int kind,
                      cudaStream_t s) {
  static_assert(sizeof(T) == 8, "the right-hand side is formed in FP64");
  const FieldGeom fg = make_field_geom(g.d, g.N[0], g.N[1], g.N[2], g.h, g.P);
  const double3 Ev = make_double3(E[0], E[1], g.d == 3 ? E[2] : 0.0);
  rhs_kernel<<<field_grid(g.P), kFieldThreads, 0, s>>>(static_cast<double2*>(b), tab, g, fg, Ev, kind);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_rhs<double>(void*, const double2*, const Geometry&, const double*, int,
                                       cudaStream_t);

// ---------------------------------------------------------------------------
// Gram matrix on Z_N (Lemma FD_matrix_full): for admissible fields
// v_i = E_i + x_i (E_i the i-th unit load),
//   X_ij = Re sum_{k in Z_N} (A v_i)^(k) . conj v_j(k),
// where (A v_i)^(k) = a^(k) E_i + y_i(k) and y_i is the operator output of x_i
// before the projection (pad, inverse transform, A_M, forward transform,
// truncation to Z_N).  v_j vanishes outside Z_N, so this is the exact energy
// the double-grid evaluation gives.
//
// At high contrast the terms of this sum cancel (the field is small where the
// coefficient is large), so the sum is carried as an unevaluated pair
// hi + lo of doubles (Knuth's TwoSum, error-free): every product is rounded
// once and the sum of the rounded products is exact up to one final rounding,
// per thread, across a warp, across a block and across blocks (in block
// order).
// ---------------------------------------------------------------------------
struct DD {
  double hi, lo;
};
// hi + lo = a + b exactly (TwoSum)
__device__ __forceinline__ DD two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  const double err = (a - (s - bb)) + (b - bb);
  return DD{s, err};
}
__device__ __forceinline__ void dd_add(DD& acc, double x) {
  const DD t = two_sum(acc.hi, x);
  acc.hi = t.hi;
  acc.lo += t.lo;
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  DD t = two_sum(a.hi, b.hi);
  t.lo += a.lo + b.lo;
  return two_sum(t.hi, t.lo);
}
__device__ __forceinline__ DD dd_warp_sum(DD v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DD w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, w);
  }
  return v;
}
// Block sum of one pair per thread (valid in thread 0); barriers inside.
__device__ __forceinline__ DD dd_block_sum(DD v, double* sh /* 64 doubles */) {
  v = dd_warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sh[wid] = v.hi;
    sh[32 + wid] = v.lo;
  }
  __syncthreads();
  DD r{0.0, 0.0};
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    if (lane < nw) r = DD{sh[lane], sh[32 + lane]};
    r = dd_warp_sum(r);
  }
  return r;
}

template <int D>
__global__ void __launch_bounds__(kFieldThreads) gram_zn_kernel(GramZnArgs ga, const double2* __restrict__ tab,
                                                                Geometry g, FieldGeom fg, double* partials) {
  __shared__ double red[64];
  const int Ld = g.N[D - 1];
  const int L1 = 2 * g.N[1] - 1;
  DD acc[D * D];
#pragma unroll
  for (int q = 0; q < D * D; ++q) acc[q] = DD{0.0, 0.0};
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int k[3];
    int j;
    kvec(fg, e, k, j);
    const double wt = (j == 0) ? 1.0 : 2.0;   // exact scaling: the mirrored half
    int64_t ti;
    if (D == 2) ti = static_cast<int64_t>(k[0] + g.N[0] - 1) * Ld + j;
    else ti = (static_cast<int64_t>(k[0] + g.N[0] - 1) * L1 + (k[1] + g.N[1] - 1)) * Ld + j;
    const double2 a = tab[ti];
    double2 v[D][D], y[D][D];   // [field][component]
#pragma unroll
    for (int f = 0; f < D; ++f)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        v[f][c] = ga.v[f][c * fg.P + e];
        y[f][c] = ga.y[f][c * fg.P + e];
      }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      // (A v_i)^(k): y_i plus a^(k) in component i
      double2 av[D];
#pragma unroll
      for (int c = 0; c < D; ++c) av[c] = (c == i) ? make_double2(y[i][c].x + a.x, y[i][c].y + a.y) : y[i][c];
#pragma unroll
      for (int jf = 0; jf < D; ++jf)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          dd_add(acc[i * D + jf], wt * (av[c].x * v[jf][c].x));
          dd_add(acc[i * D + jf], wt * (av[c].y * v[jf][c].y));
        }
    }
  }
  const int64_t nb = gridDim.x;
#pragma unroll
  for (int q = 0; q < D * D; ++q) {
    const DD bs = dd_block_sum(acc[q], red);
    if (threadIdx.x == 0) {
      partials[(2 * static_cast<int64_t>(q)) * nb + blockIdx.x] = bs.hi;
      partials[(2 * static_cast<int64_t>(q) + 1) * nb + blockIdx.x] = bs.lo;
    }
  }
}

__global__ void __launch_bounds__(kFieldThreads) gram_zn_final(const double* __restrict__ partials, int nb, int dd,
                                                               double* out) {
  __shared__ double red[64];
  for (int q = 0; q < dd; ++q) {
    DD s{0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      s = dd_add(s, DD{partials[(2 * static_cast<int64_t>(q)) * nb + b],
                       partials[(2 * static_cast<int64_t>(q) + 1) * nb + b]});
    s = dd_block_sum(s, red);
    if (threadIdx.x == 0) out[q] = s.hi + s.lo;
  }
}

ghb_status launch_gram_zn(const GramZnArgs& ga, const double2* tab, const Geometry& g, double* partials,
                          int max_partials, double* out, cudaStream_t s) {
  const FieldGeom fg = make_field_geom(g.d, g.N[0], g.N[1], g.N[2], g.h, g.P);
  const int dd = g.d * g.d;
  int nb = field_grid(g.P);
  if (2 * nb * dd > max_partials) nb = max_partials / (2 * dd);   // hi and lo per block and entry
  if (g.d == 2) gram_zn_kernel<2><<<nb, kFieldThreads, 0, s>>>(ga, tab, g, fg, partials);
  else gram_zn_kernel<3><<<nb, kFieldThreads, 0, s>>>(ga, tab, g, fg, partials);
  GHB_CUDA_TRY(cudaGetLastError());
  gram_zn_final<<<1, kFieldThreads, 0, s>>>(partials, nb, dd, out);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

namespace {
// Blocks of one vector-operation launch: the field's grid, but at most the
// blocks of this kernel that are resident on the device at once (the loops
// stride over the field, so one full wave does the work without a partly
// filled second wave: the FP32 projection kernel holds 5 blocks per SM, and
// its 1216-block grid ran 1.6 waves).  The count is taken once per process
// (one device model).
template <typename T, int OP>
int64_t one_wave(int64_t want) {
  static std::atomic<int> wave{0};
  int w = wave.load(std::memory_order_relaxed);
  if (w == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel<T, OP>, kFieldThreads, 0) != cudaSuccess ||
        sms < 1 || per_sm < 1)
      return want;
    w = sms * per_sm;
    wave.store(w, std::memory_order_relaxed);
  }
  return std::min<int64_t>(want, w);
}

template <typename T, int OP>
ghb_status launch_one(const CgItem& it, cudaStream_t s) {
  const int64_t nb = one_wave<T, OP>(it.nblocks);
  cg_kernel<T, OP><<<static_cast<unsigned>(nb), kFieldThreads, 0, s>>>(it);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
CgItem make_item(const FieldGeom& fg) {
  CgItem it{};
  it.fg = fg;
  it.nblocks = field_grid(fg.P);
  return it;
}
}  // namespace

int64_t cg_blocks(const FieldGeom& fg) { return field_grid(fg.P); }

template <typename T>
ghb_status launch_project(void* y, const void* w, const FieldGeom& fg, int kind, cudaStream_t s) {
  CgItem it = make_item(fg);
  it.q = y;
  it.w = w;
  it.kind = kind;
  return launch_one<T, CG_PROJECT>(it, s);
}
template ghb_status launch_project<double>(void*, const void*, const FieldGeom&, int, cudaStream_t);
template ghb_status launch_project<float>(void*, const void*, const FieldGeom&, int, cudaStream_t);

template <typename T>
ghb_status launch_cg_init(void* x, void* r, void* p, const void* b, const FieldGeom& fg, CgState* st,
                          double* partials, double tol, int maxiter, cudaStream_t s) {
  CgItem it = make_item(fg);
  it.x = x;
  it.r = r;
  it.p = p;
  it.b = b;
  it.st = st;
  it.partials = partials;
  it.tol = tol;
  it.maxiter = maxiter;
  return launch_one<T, CG_INIT>(it, s);
}
template ghb_status launch_cg_init<double>(void*, void*, void*, const void*, const FieldGeom&,
                                           CgState*, double*, double, int, cudaStream_t);
template ghb_status launch_cg_init<float>(void*, void*, void*, const void*, const FieldGeom&,
                                          CgState*, double*, double, int, cudaStream_t);

template <typename T>
ghb_status launch_project_dot(void* q, const void* w, const void* p, const FieldGeom& fg, int kind,
                              CgState* st, double* partials, cudaStream_t s) {
  CgItem it = make_item(fg);
  it.q = q;
  it.w = w;
  it.p = const_cast<void*>(p);
  it.kind = kind;
  it.st = st;
  it.partials = partials;
  return launch_one<T, CG_PROJECT_DOT>(it, s);
}
template ghb_status launch_project_dot<double>(void*, const void*, const void*, const FieldGeom&,
                                               int, CgState*, double*, cudaStream_t);
template ghb_status launch_project_dot<float>(void*, const void*, const void*, const FieldGeom&, int,
                                              CgState*, double*, cudaStream_t);

template <typename T>
ghb_status launch_update(void* x, void* r, const void* p, const void* q, const FieldGeom& fg,
                         CgState* st, double* partials, cudaStream_t s) {
  CgItem it = make_item(fg);
  it.x = x;
  it.r = r;
  it.p = const_cast<void*>(p);
  it.q = const_cast<void*>(q);
  it.st = st;
  it.partials = partials;
  return launch_one<T, CG_UPDATE>(it, s);
}
template ghb_status launch_update<double>(void*, void*, const void*, const void*, const FieldGeom&,
                                          CgState*, double*, cudaStream_t);
template ghb_status launch_update<float>(void*, void*, const void*, const void*, const FieldGeom&,
                                         CgState*, double*, cudaStream_t);

ghb_status launch_residual(double2* r, const double2* b, const double2* y, const FieldGeom& fg,
                           CgState* st, double* partials, cudaStream_t s) {
  CgItem it = make_item(fg);
  it.r = r;
  it.b = b;
  it.w = y;
  it.st = st;
  it.partials = partials;
  return launch_one<double, CG_RESIDUAL>(it, s);
}

ghb_status launch_to_f32(float2* dst, const double2* src, const FieldGeom& fg, cudaStream_t s) {
  CgItem it = make_item(fg);
  it.q = dst;
  it.w = src;
  return launch_one<double, CG_TO_F32>(it, s);
}

ghb_status launch_accum_f32(double2* x, const double2* base, const float2* dx, const FieldGeom& fg,
                            cudaStream_t s) {
  CgItem it = make_item(fg);
  it.x = x;
  it.w = base;
  it.p = const_cast<float2*>(dx);
  return launch_one<double, CG_ACCUM>(it, s);
}

template <typename T>
ghb_status launch_cg_batch(int op, const CgItem* items, int n, int64_t blocks, cudaStream_t s) {
  const unsigned g = static_cast<unsigned>(blocks);
  switch (op) {
    case CG_INIT: cg_kernel_batch<T, CG_INIT><<<g, kFieldThreads, 0, s>>>(items, n); break;
    case CG_PROJECT_DOT: cg_kernel_batch<T, CG_PROJECT_DOT><<<g, kFieldThreads, 0, s>>>(items, n); break;
    case CG_UPDATE: cg_kernel_batch<T, CG_UPDATE><<<g, kFieldThreads, 0, s>>>(items, n); break;
    case CG_PROJECT: cg_kernel_batch<T, CG_PROJECT><<<g, kFieldThreads, 0, s>>>(items, n); break;
    case CG_RESIDUAL: cg_kernel_batch<double, CG_RESIDUAL><<<g, kFieldThreads, 0, s>>>(items, n); break;
    case CG_TO_F32: cg_kernel_batch<double, CG_TO_F32><<<g, kFieldThreads, 0, s>>>(items, n); break;
    case CG_ACCUM: cg_kernel_batch<double, CG_ACCUM><<<g, kFieldThreads, 0, s>>>(items, n); break;
    default: set_error("internal: bad batched CG op"); return GHB_ERR_INVALID;
  }
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_cg_batch<double>(int, const CgItem*, int, int64_t, cudaStream_t);
template ghb_status launch_cg_batch<float>(int, const CgItem*, int, int64_t, cudaStream_t);

ghb_status launch_to_f32_real(float* dst, const double* src, int64_t n, cudaStream_t s) {
  to_f32_real_kernel<<<field_grid(n), kFieldThreads, 0, s>>>(dst, src, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

ghb_status launch_add_constant(double2* v, const double2* e, const FieldGeom& fg, const double* E,
                               cudaStream_t s) {
  int64_t e0;
  if (fg.d == 2) e0 = static_cast<int64_t>((fg.N[0] - 1) / 2) * fg.h;
  else e0 = (static_cast<int64_t>((fg.N[0] - 1) / 2) * fg.N[1] + (fg.N[1] - 1) / 2) * fg.h;
  const double3 Ev = make_double3(E[0], E[1], fg.d == 3 ? E[2] : 0.0);
  add_constant_kernel<<<field_grid(fg.P), kFieldThreads, 0, s>>>(v, e, fg, Ev, e0);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}


// ---------------------------------------------------------------------------
// GaNi data: point samples of the coefficient (eq. approx_bilin)
// ---------------------------------------------------------------------------
namespace {

// x^k = k / N per axis; a point belongs to an inclusion when its periodic
// offset from the centre is at most the radius (disk, sphere) or at most half
// the side along every axis (box).  The arithmetic is written with explicit
// roundings (no fused multiply-add) so that the membership decisions are those
// of the same formula evaluated operation by operation in FP64.
__global__ void sample_kernel(double* out64, float* out32, Geometry g, const Incl* __restrict__ incs, int n,
                              double a0v) {
  const int d = g.d;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < g.grid;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int k[3] = {0, 0, 0};
    int64_t rem = idx;
    for (int a = d - 1; a >= 0; --a) {
      k[a] = static_cast<int>(rem % g.N[a]);
      rem /= g.N[a];
    }
    double v = a0v;
    for (int i = 0; i < n; ++i) {
      const Incl in = incs[i];
      double dist[3] = {0.0, 0.0, 0.0};
      for (int a = 0; a < d; ++a) {
        const double t = __dsub_rn(__ddiv_rn(static_cast<double>(k[a]), static_cast<double>(g.N[a])), in.c[a]);
        dist[a] = __dsub_rn(t, rint(t));
      }
      bool inside;
      if (in.shape == GHB_BOX) {
        inside = true;
        for (int a = 0; a < d; ++a) inside = inside && (fabs(dist[a]) <= 0.5 * in.s[a]);
      } else {
        double s = __dmul_rn(dist[0], dist[0]);
        for (int a = 1; a < d; ++a) s = __dadd_rn(s, __dmul_rn(dist[a], dist[a]));
        inside = s <= __dmul_rn(in.s[0], in.s[0]);
      }
      if (inside) v = in.v;
    }
    out64[idx] = v;
    out32[idx] = static_cast<float>(v);
  }
}

__global__ void scale_kernel(double2* v, double s, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double2 z = v[i];
    v[i] = make_double2(s * z.x, s * z.y);
  }
}

unsigned elementwise_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return static_cast<unsigned>(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

ghb_status launch_sample_values(double* out64, float* out32, const Geometry& g, const Incl* incs, int n,
                                double a0v, cudaStream_t s) {
  sample_kernel<<<elementwise_blocks(g.grid), 256, 0, s>>>(out64, out32, g, incs, n, a0v);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

ghb_status launch_scale(double2* v, double sc, int64_t n, cudaStream_t s) {
  scale_kernel<<<elementwise_blocks(n), 256, 0, s>>>(v, sc, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}


// ---------------------------------------------------------------------------
// prolongation Z_Nc -> Z_Nf and y += a x
// ---------------------------------------------------------------------------
namespace {

__global__ void prolong_kernel(double2* xf, FieldGeom ff, const double2* __restrict__ xc, FieldGeom fc) {
  const int d = ff.d;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < ff.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // fine index (i_1 .. i_{d-1} centred, j on the half axis) -> coarse index
    int64_t rem = e;
    const int j = static_cast<int>(rem % ff.h);
    rem /= ff.h;
    bool in = j < fc.h;
    int64_t ec = j;
    int64_t stride = fc.h;
    for (int a = d - 2; a >= 0; --a) {
      const int i = static_cast<int>(rem % ff.N[a]);
      rem /= ff.N[a];
      const int k = i - (ff.N[a] - 1) / 2;             // frequency
      const int ic = k + (fc.N[a] - 1) / 2;
      in = in && ic >= 0 && ic < fc.N[a];
      ec += static_cast<int64_t>(ic) * stride;
      stride *= fc.N[a];
    }
    for (int c = 0; c < d; ++c) xf[c * ff.P + e] = in ? xc[c * fc.P + ec] : make_double2(0.0, 0.0);
  }
}

__global__ void axpy_kernel(double2* y, const double2* __restrict__ x, double a, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double2 u = x[i], v = y[i];
    y[i] = make_double2(v.x + a * u.x, v.y + a * u.y);
  }
}

}  // namespace

ghb_status launch_prolong(double2* xf, const FieldGeom& ff, const double2* xc, const FieldGeom& fc,
                          cudaStream_t s) {
  prolong_kernel<<<elementwise_blocks(ff.P), 256, 0, s>>>(xf, ff, xc, fc);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

ghb_status launch_axpy(double2* y, const double2* x, double a, int64_t n, cudaStream_t s) {
  axpy_kernel<<<elementwise_blocks(n), 256, 0, s>>>(y, x, a, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}


// ---------------------------------------------------------------------------
// coefficient table of a pixel image (Lemma grid_compos)
// ---------------------------------------------------------------------------
namespace {

__device__ double pixel_sinc(int m, int P) {   // sinc(m / P) = sin(pi m / P) / (pi m / P)
  if (m == 0) return 1.0;
  const double x = static_cast<double>(m) / static_cast<double>(P);
  return sinpi(x) / (3.141592653589793238462643383279502884 * x);
}

__global__ void image_table_kernel(double2* tab, Geometry g, const double2* __restrict__ chat, int3 P3) {
  const int d = g.d;
  const int P[3] = {P3.x, P3.y, P3.z};
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < g.table;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // half table: leading axes centred on Z_{2N_a - 1}, last axis m_d = 0 .. N_d - 1
    int m[3] = {0, 0, 0};
    int64_t rem = e;
    m[d - 1] = static_cast<int>(rem % g.N[d - 1]);
    rem /= g.N[d - 1];
    for (int a = d - 2; a >= 0; --a) {
      const int L = 2 * g.N[a] - 1;
      m[a] = static_cast<int>(rem % L) - (g.N[a] - 1);
      rem /= L;
    }
    int64_t idx = 0;
    double f = 1.0;
    for (int a = 0; a < d; ++a) {
      int i = (m[a] + (P[a] - 1) / 2) % P[a];
      if (i < 0) i += P[a];
      idx = idx * P[a] + i;
      f *= pixel_sinc(m[a], P[a]);
    }
    const double2 cv = chat[idx];
    tab[e] = make_double2(f * cv.x, f * cv.y);
  }
}

}  // namespace

ghb_status launch_image_table(double2* tab, const Geometry& g, const double2* chat, const int* P, cudaStream_t s) {
  image_table_kernel<<<elementwise_blocks(g.table), 256, 0, s>>>(tab, g, chat, make_int3(P[0], P[1], P[2]));
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}


// ---------------------------------------------------------------------------
// reduced Ga operator (Lemma reduce_grid): sub-grids and DFT shifts
// ---------------------------------------------------------------------------
namespace {

__global__ void subgrid_kernel(double* out64, float* out32, const double* __restrict__ grid, Geometry g,
                               int shift, int64_t n) {
  const int d = g.d;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t rem = e, idx = 0, stride = 1;
    int r[3] = {0, 0, 0};
    for (int a = d - 1; a >= 0; --a) {
      r[a] = static_cast<int>(rem % g.N[a]);
      rem /= g.N[a];
    }
    for (int a = d - 1; a >= 0; --a) {
      const int sa = (shift >> a) & 1;
      int m = 2 * r[a] - sa;
      if (m < 0) m += g.M[a];
      idx += static_cast<int64_t>(m) * stride;
      stride *= g.M[a];
    }
    const double v = grid[idx];
    out64[e] = v;
    out32[e] = static_cast<float>(v);
  }
}

template <typename T>
__global__ void phase_kernel(typename CT<T>::type* y, const typename CT<T>::type* __restrict__ x, FieldGeom fg,
                             int shift, int sign, T a, T b, const CgState* st) {
  using C = typename CT<T>::type;
  if (st != nullptr && st->done != RUNNING) return;
  const int d = fg.d;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t rem = e;
    const int j = static_cast<int>(rem % fg.h);
    rem /= fg.h;
    // sum_a s_a m_a / N_a, m the frequency (leading axes centred, last axis j)
    T t = ((shift >> (d - 1)) & 1) ? static_cast<T>(j) / static_cast<T>(fg.N[d - 1]) : T(0);
    for (int ax = d - 2; ax >= 0; --ax) {
      const int i = static_cast<int>(rem % fg.N[ax]);
      rem /= fg.N[ax];
      if ((shift >> ax) & 1) t += static_cast<T>(i - (fg.N[ax] - 1) / 2) / static_cast<T>(fg.N[ax]);
    }
    T sn, cs;
    if constexpr (sizeof(T) == 8) sincospi(static_cast<double>(sign) * t, &sn, &cs);
    else sincospif(static_cast<float>(sign) * t, &sn, &cs);
    for (int c = 0; c < d; ++c) {
      const C xv = x[c * fg.P + e];
      const C rot = mk(b * (cs * xv.x - sn * xv.y), b * (cs * xv.y + sn * xv.x));
      if (a == T(0)) {
        y[c * fg.P + e] = rot;
      } else {
        const C yv = y[c * fg.P + e];
        y[c * fg.P + e] = mk(a * yv.x + rot.x, a * yv.y + rot.y);
      }
    }
  }
}

}  // namespace

ghb_status launch_subgrid(double* out64, float* out32, const double* grid64, const Geometry& g, int shift,
                          cudaStream_t s) {
  int64_t n = 1;
  for (int a = 0; a < g.d; ++a) n *= g.N[a];
  subgrid_kernel<<<elementwise_blocks(n), 256, 0, s>>>(out64, out32, grid64, g, shift, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

template <typename T>
ghb_status launch_phase(void* y, const void* x, const FieldGeom& fg, int shift, int sign, double a, double b,
                        const CgState* st, cudaStream_t s) {
  using C = typename CT<T>::type;
  phase_kernel<T><<<elementwise_blocks(fg.P), 256, 0, s>>>(static_cast<C*>(y), static_cast<const C*>(x), fg, shift,
                                                           sign, static_cast<T>(a), static_cast<T>(b), st);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_phase<double>(void*, const void*, const FieldGeom&, int, int, double, double,
                                         const CgState*, cudaStream_t);
template ghb_status launch_phase<float>(void*, const void*, const FieldGeom&, int, int, double, double,
                                        const CgState*, cudaStream_t);

}  // namespace ghb
