// Field-level kernels: coefficient tables, right-hand sides, projections and
// the conjugate-gradient vector updates with their FP64 reductions.
//
// Fields are half spectra on Z_N (see ghb.h): x[c][i_1]..[i_{d-1}][j].  The
// inner product of the paper's complex space (Section 5.1,
// (u, v) = sum_{k in Z_N} u(k).conj v(k)) is evaluated on the half spectrum as
// sum_k w_k Re(u(k).conj v(k)) with weight w_k = 1 on the plane k_d = 0 and 2
// elsewhere (each stored k_d > 0 stands for k and -k).
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

__device__ __forceinline__ void kvec(const FieldGeom& g, int64_t e, int k[3], int& j) {
  if (g.d == 2) {
    const int64_t i1 = e / g.h;
    j = static_cast<int>(e - i1 * g.h);
    k[0] = static_cast<int>(i1) - (g.N[0] - 1) / 2;
    k[1] = j;
    k[2] = 0;
  } else {
    const int64_t plane = static_cast<int64_t>(g.N[1]) * g.h;
    const int64_t i1 = e / plane;
    const int64_t rem = e - i1 * plane;
    const int64_t i2 = rem / g.h;
    j = static_cast<int>(rem - i2 * g.h);
    k[0] = static_cast<int>(i1) - (g.N[0] - 1) / 2;
    k[1] = static_cast<int>(i2) - (g.N[1] - 1) / 2;
    k[2] = j;
  }
}

// Index of the entry holding -k for an entry on the plane k_d = 0 (where both
// k and -k are stored); -1 elsewhere.
__device__ __forceinline__ int64_t mirror_index(const FieldGeom& g, int64_t e, int j) {
  if (j != 0) return -1;
  if (g.d == 2) {
    const int64_t i1 = e / g.h;
    return (g.N[0] - 1 - i1) * g.h;
  }
  const int64_t i12 = e / g.h;
  const int64_t i1 = i12 / g.N[1];
  const int64_t i2 = i12 - i1 * g.N[1];
  return ((g.N[0] - 1 - i1) * g.N[1] + (g.N[1] - 1 - i2)) * g.h;
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
  sx /= kk;
  sy /= kk;
  for (int c = 0; c < d; ++c) {
    const C pe = mk(kv[c] * sx, kv[c] * sy);
    q[c] = (kind == GHB_PRIMAL) ? pe : mk(w[c].x - pe.x, w[c].y - pe.y);
  }
}

// Grid-wide sum: partial per block, the last block to finish adds the
// partials in block order.  Returns true in thread 0 of that block with *total.
__device__ bool grid_sum_last(double v, double* partials, unsigned int* ticket, double* total) {
  __shared__ double red[32];
  __shared__ bool last;
  const double bs = block_sum(v, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(&partials[b]);
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
    return r * j1(2.0 * kPi * r * rho) / rho;
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

__global__ void coeff_kernel(double2* tab, Geometry g, const Incl* incs, int n, double a0v) {
  const int d = g.d;
  const int L0 = 2 * g.N[0] - 1;
  const int L1 = (d == 3) ? 2 * g.N[1] - 1 : g.N[1];
  const int Ld = g.N[d - 1];   // half of 2N_d - 1: n_d = 0..N_d-1
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < g.table;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int nv[3] = {0, 0, 0};
    if (d == 2) {
      const int64_t i0 = e / Ld;
      nv[0] = static_cast<int>(i0) - (g.N[0] - 1);
      nv[1] = static_cast<int>(e - i0 * Ld);
    } else {
      const int64_t pl = static_cast<int64_t>(L1) * Ld;
      const int64_t i0 = e / pl;
      const int64_t rem = e - i0 * pl;
      const int64_t i1 = rem / Ld;
      nv[0] = static_cast<int>(i0) - (g.N[0] - 1);
      nv[1] = static_cast<int>(i1) - (g.N[1] - 1);
      nv[2] = static_cast<int>(rem - i1 * Ld);
    }
    (void)L0;
    double re = (nv[0] == 0 && nv[1] == 0 && nv[2] == 0) ? a0v : 0.0;
    double im = 0.0;
    for (int i = 0; i < n; ++i) {
      const Incl in = incs[i];
      // exp(-2 pi i n.x_i): reduce n.x_i to [-1/2, 1/2] before the sincos
      double t = 0.0;
      for (int a = 0; a < d; ++a) t = fma(static_cast<double>(nv[a]), in.c[a], t);
      t -= rint(t);
      double s, c;
      sincospi(2.0 * t, &s, &c);
      const double f = in.dv * shape_coeff(in, d, nv);
      re += f * c;
      im -= f * s;
    }
    tab[e] = make_double2(re, im);
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

// y = G w (with the Hermitian part taken on k_d = 0); y must not alias w.
template <typename T>
__global__ void project_kernel(typename CT<T>::type* y, const typename CT<T>::type* w, FieldGeom fg,
                               int kind) {
  using C = typename CT<T>::type;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int k[3];
    int j;
    kvec(fg, e, k, j);
    const int64_t em = mirror_index(fg, e, j);
    C wv[3], q[3];
    for (int c = 0; c < fg.d; ++c) wv[c] = hermitian_part(w, fg.P, c, e, em);
    project_vec<T>(fg.d, k, kind, wv, q);
    for (int c = 0; c < fg.d; ++c) y[c * fg.P + e] = q[c];
  }
}

template <typename T>
__global__ void cg_init_kernel(typename CT<T>::type* x, typename CT<T>::type* r,
                               typename CT<T>::type* p, const typename CT<T>::type* b, FieldGeom fg,
                               CgState* st, double* partials, double tol, int maxiter) {
  using C = typename CT<T>::type;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int k[3];
    int j;
    kvec(fg, e, k, j);
    const double wt = (j == 0) ? 1.0 : 2.0;
    for (int c = 0; c < fg.d; ++c) {
      const int64_t i = c * fg.P + e;
      const C bv = b[i];
      x[i] = mk(T(0), T(0));
      p[i] = mk(T(0), T(0));
      r[i] = bv;
      acc += wt * (double(bv.x) * bv.x + double(bv.y) * bv.y);
    }
  }
  double tot;
  if (grid_sum_last(acc, partials, &st->ticket, &tot)) {
    st->bb = tot;
    st->rr = tot;
    st->tol2 = tol * tol * tot;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->pq = 0.0;
    st->iter = 0;
    st->maxiter = maxiter;
    st->done = (tot == 0.0) ? CONVERGED : RUNNING;
  }
}

// q = G w, <p, q>; the last block forms alpha = <r, r> / <p, A p>.
template <typename T>
__global__ void project_dot_kernel(typename CT<T>::type* q, const typename CT<T>::type* w,
                                   const typename CT<T>::type* p, FieldGeom fg, int kind,
                                   CgState* st, double* partials) {
  using C = typename CT<T>::type;
  if (st->done != RUNNING) return;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int k[3];
    int j;
    kvec(fg, e, k, j);
    const double wt = (j == 0) ? 1.0 : 2.0;
    const int64_t em = mirror_index(fg, e, j);
    C wv[3], qv[3];
    for (int c = 0; c < fg.d; ++c) wv[c] = hermitian_part(w, fg.P, c, e, em);
    project_vec<T>(fg.d, k, kind, wv, qv);
    double s = 0.0;
    for (int c = 0; c < fg.d; ++c) {
      q[c * fg.P + e] = qv[c];
      const C pv = p[c * fg.P + e];
      s += double(pv.x) * qv[c].x + double(pv.y) * qv[c].y;
    }
    acc += wt * s;
  }
  double tot;
  if (grid_sum_last(acc, partials, &st->ticket, &tot)) {
    st->pq = tot;
    if (!(tot > 0.0) || !isfinite(tot)) {
      st->done = BREAKDOWN;
      st->alpha = 0.0;
    } else {
      st->alpha = st->rr / tot;
    }
  }
}

// x += alpha p, r -= alpha q, <r, r>; the last block forms beta and the stop test.
template <typename T>
__global__ void update_kernel(typename CT<T>::type* x, typename CT<T>::type* r,
                              const typename CT<T>::type* p, const typename CT<T>::type* q,
                              FieldGeom fg, CgState* st, double* partials) {
  using C = typename CT<T>::type;
  if (st->done != RUNNING) return;
  const T al = static_cast<T>(st->alpha);
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i1 = (fg.d == 2) ? e / fg.h : e / (static_cast<int64_t>(fg.N[1]) * fg.h);
    (void)i1;
    const int j = static_cast<int>(e % fg.h);
    const double wt = (j == 0) ? 1.0 : 2.0;
    for (int c = 0; c < fg.d; ++c) {
      const int64_t i = c * fg.P + e;
      const C pv = p[i], qv = q[i];
      C xv = x[i], rv = r[i];
      xv = mk(xv.x + al * pv.x, xv.y + al * pv.y);
      rv = mk(rv.x - al * qv.x, rv.y - al * qv.y);
      x[i] = xv;
      r[i] = rv;
      acc += wt * (double(rv.x) * rv.x + double(rv.y) * rv.y);
    }
  }
  double tot;
  if (grid_sum_last(acc, partials, &st->ticket, &tot)) {
    const double rr_old = st->rr;
    st->beta = tot / rr_old;
    st->rr = tot;
    st->iter += 1;
    if (!isfinite(tot)) st->done = BREAKDOWN;
    else if (tot <= st->tol2) st->done = CONVERGED;
    else if (st->iter >= st->maxiter) st->done = MAXITER;
  }
}

__global__ void residual_kernel(double2* r, const double2* b, const double2* y, FieldGeom fg,
                                CgState* st, double* partials) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < fg.P;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(e % fg.h);
    const double wt = (j == 0) ? 1.0 : 2.0;
    for (int c = 0; c < fg.d; ++c) {
      const int64_t i = c * fg.P + e;
      const double2 rv = make_double2(b[i].x - y[i].x, b[i].y - y[i].y);
      r[i] = rv;
      acc += wt * (rv.x * rv.x + rv.y * rv.y);
    }
  }
  double tot;
  if (grid_sum_last(acc, partials, &st->ticket, &tot)) st->rr = tot;
}

__global__ void to_f32_kernel(float2* dst, const double2* src, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[i] = make_float2(static_cast<float>(src[i].x), static_cast<float>(src[i].y));
}

__global__ void accum_f32_kernel(double2* x, const float2* dx, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] = make_double2(x[i].x + static_cast<double>(dx[i].x), x[i].y + static_cast<double>(dx[i].y));
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
ghb_status launch_coeff_table(double2* tab, const Geometry& g, const Incl* incs, int n, double a0v,
                              cudaStream_t s) {
  coeff_kernel<<<field_grid(g.table), kFieldThreads, 0, s>>>(tab, g, incs, n, a0v);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

template <typename T>
ghb_status launch_rhs(void* b, const double2* tab, const Geometry& g, const double* E, int kind,
                      cudaStream_t s) {
  static_assert(sizeof(T) == 8, "the right-hand side is formed in FP64");
  FieldGeom fg{g.d, {g.N[0], g.N[1], g.N[2]}, g.h, g.P};
  const double3 Ev = make_double3(E[0], E[1], g.d == 3 ? E[2] : 0.0);
  rhs_kernel<<<field_grid(g.P), kFieldThreads, 0, s>>>(static_cast<double2*>(b), tab, g, fg, Ev, kind);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_rhs<double>(void*, const double2*, const Geometry&, const double*, int,
                                       cudaStream_t);

template <typename T>
ghb_status launch_project(void* y, const void* w, const FieldGeom& fg, int kind, cudaStream_t s) {
  using C = typename CT<T>::type;
  project_kernel<T><<<field_grid(fg.P), kFieldThreads, 0, s>>>(static_cast<C*>(y),
                                                                static_cast<const C*>(w), fg, kind);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_project<double>(void*, const void*, const FieldGeom&, int, cudaStream_t);
template ghb_status launch_project<float>(void*, const void*, const FieldGeom&, int, cudaStream_t);

template <typename T>
ghb_status launch_cg_init(void* x, void* r, void* p, const void* b, const FieldGeom& fg, CgState* st,
                          double* partials, double tol, int maxiter, cudaStream_t s) {
  using C = typename CT<T>::type;
  cg_init_kernel<T><<<field_grid(fg.P), kFieldThreads, 0, s>>>(
      static_cast<C*>(x), static_cast<C*>(r), static_cast<C*>(p), static_cast<const C*>(b), fg, st,
      partials, tol, maxiter);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_cg_init<double>(void*, void*, void*, const void*, const FieldGeom&,
                                           CgState*, double*, double, int, cudaStream_t);
template ghb_status launch_cg_init<float>(void*, void*, void*, const void*, const FieldGeom&,
                                          CgState*, double*, double, int, cudaStream_t);

template <typename T>
ghb_status launch_project_dot(void* q, const void* w, const void* p, const FieldGeom& fg, int kind,
                              CgState* st, double* partials, cudaStream_t s) {
  using C = typename CT<T>::type;
  project_dot_kernel<T><<<field_grid(fg.P), kFieldThreads, 0, s>>>(
      static_cast<C*>(q), static_cast<const C*>(w), static_cast<const C*>(p), fg, kind, st, partials);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_project_dot<double>(void*, const void*, const void*, const FieldGeom&,
                                               int, CgState*, double*, cudaStream_t);
template ghb_status launch_project_dot<float>(void*, const void*, const void*, const FieldGeom&, int,
                                              CgState*, double*, cudaStream_t);

template <typename T>
ghb_status launch_update(void* x, void* r, const void* p, const void* q, const FieldGeom& fg,
                         CgState* st, double* partials, cudaStream_t s) {
  using C = typename CT<T>::type;
  update_kernel<T><<<field_grid(fg.P), kFieldThreads, 0, s>>>(
      static_cast<C*>(x), static_cast<C*>(r), static_cast<const C*>(p), static_cast<const C*>(q), fg,
      st, partials);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}
template ghb_status launch_update<double>(void*, void*, const void*, const void*, const FieldGeom&,
                                          CgState*, double*, cudaStream_t);
template ghb_status launch_update<float>(void*, void*, const void*, const void*, const FieldGeom&,
                                         CgState*, double*, cudaStream_t);

ghb_status launch_residual(double2* r, const double2* b, const double2* y, const FieldGeom& fg,
                           CgState* st, double* partials, cudaStream_t s) {
  residual_kernel<<<field_grid(fg.P), kFieldThreads, 0, s>>>(r, b, y, fg, st, partials);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

ghb_status launch_to_f32(float2* dst, const double2* src, int64_t n, cudaStream_t s) {
  to_f32_kernel<<<field_grid(n), kFieldThreads, 0, s>>>(dst, src, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

ghb_status launch_accum_f32(double2* x, const float2* dx, int64_t n, cudaStream_t s) {
  accum_f32_kernel<<<field_grid(n), kFieldThreads, 0, s>>>(x, dx, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

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

}  // namespace ghb
