// C ABI of the ghb library: context, coefficient set-up, operator, CG solves
// (FP64 and mixed FP32/FP64), Gram energies and bounds.  See include/ghb.h.
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ghb_internal.cuh"

namespace ghb {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

}  // namespace ghb

using namespace ghb;

// Device buffers of one precision.
template <typename C>
struct Work {
  C* x = nullptr;
  C* r = nullptr;
  C* p = nullptr;
  C* q = nullptr;
  C* w = nullptr;
  C* T1 = nullptr;
  C* T2 = nullptr;
  C* s1 = nullptr;   // reduced operator: the shifted direction and one shift's image
  C* s2 = nullptr;
};

// One Galerkin operator: the geometry of its transforms, a plan per axis and
// its real multiplier on the transform grid.  `ga`: Algorithm 2 on the double
// grid M with the exact values A_M (eq. MBA_GA).  `gani`: Algorithm 1, the
// same passes on the N grid (M = N) with the point samples of a (Def. GaNi).
struct OpView {
  Geometry g{};
  const FftPlan* plan[3] = {nullptr, nullptr, nullptr};
  double* grid64[2] = {nullptr, nullptr};
  float* grid32[2] = {nullptr, nullptr};
};

struct ghb_ctx {
  Geometry g{};
  ghb_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  PlanHolder plan[3];
  int plan_of_axis[3] = {0, 1, 2};

  // coefficient data: [0] = a (primal), [1] = 1/a (dual)
  double2* tab[2] = {nullptr, nullptr};
  double* grid64[2] = {nullptr, nullptr};
  float* grid32[2] = {nullptr, nullptr};
  double2* tabT1 = nullptr;   // table transform intermediates
  double2* tabT2 = nullptr;
  Incl* d_incs = nullptr;
  int incs_cap = 0;

  Work<double2> w64;
  Work<float2> w32;
  double2* b64 = nullptr;      // right-hand side (FP64)
  double2* y64 = nullptr;      // FP64 operator output (outer residual)
  double2* sol[3] = {nullptr, nullptr, nullptr};   // admissible fields of ghb_bounds
  double2* gT1[3] = {nullptr, nullptr, nullptr};   // Gram intermediates per field
  double2* gT2[3] = {nullptr, nullptr, nullptr};

  CgState* st = nullptr;
  CgState* h_st = nullptr;     // pinned host mirror
  double* partials = nullptr;
  unsigned int* ticket = nullptr;
  double* d_gram = nullptr;
  double* h_gram = nullptr;    // pinned
  int64_t bytes = 0;

  // operators: the Ga one, the GaNi one (built on first use) and the one the
  // CG, operator and Gram routines act on
  OpView ga, gani;
  const OpView* op = nullptr;
  bool gani_ready = false;
  PlanHolder planN[3];
  int planN_of_axis[3] = {0, 1, 2};
  double* gridN64[2] = {nullptr, nullptr};
  float* gridN32[2] = {nullptr, nullptr};
  double a0 = 1.0;      // microstructure, for the GaNi samples
  int n_incs = 0;
  bool is_image = false;      // coefficients from a pixel image (no GaNi samples)
  // reduced form of the Ga operator (Lemma reduce_grid, Algorithm 3; needs M = 2N):
  // one N-grid view per shift s in {0,1}^d with the double-grid values at 2r - s
  int form = GHB_FORM_DOUBLE_GRID;
  bool red_ready = false;
  OpView red[8];
  double* redgrid64[2] = {nullptr, nullptr};
  float* redgrid32[2] = {nullptr, nullptr};
  double* d_hist = nullptr;   // energy decrease along CG iterates (bound tracking)
  int hist_cap = 0;

  // optional per-launch CUDA-event timing (ghb_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev;   // 2 per record
  std::vector<int> rec_cls;
  int nrec = 0;
};

namespace {

template <typename P>
ghb_status dmalloc(ghb_ctx* c, P** ptr, int64_t count) {
  const size_t bytes = sizeof(P) * static_cast<size_t>(count > 0 ? count : 1);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GHB_ERR_OOM : GHB_ERR_CUDA;
  }
  c->bytes += static_cast<int64_t>(bytes);
  return GHB_OK;
}

#define TRY(expr)                      \
  do {                                 \
    ghb_status s__ = (expr);           \
    if (s__ != GHB_OK) return s__;     \
  } while (0)

FieldGeom fgeom(const Geometry& g) { return make_field_geom(g.d, g.N[0], g.N[1], g.N[2], g.h, g.P); }

const FftPlan& plan_of(const ghb_ctx* c, int axis) { return c->plan[c->plan_of_axis[axis]].plan; }

// Kernel classes for ghb_profile_read: class id = 2 * kind-of-launch + (FP32 ? 1 : 0).
enum ProfKind {
  PK_COEFF = 0,     // coefficient table and its transform to the double grid
  PK_COL1_INV_PU,   // axis-1 inverse pass fused with p = r + beta p (CG)
  PK_COL1_INV,      // axis-1 inverse pass (operator, Gram)
  PK_COL2_INV,      // axis-2 inverse pass (d = 3)
  PK_ROW,           // last-axis pass: C2R, multiply by A_M, R2C
  PK_COL2_FWD,      // axis-2 forward pass (d = 3)
  PK_COL1_FWD,      // axis-1 forward pass, truncation to Z_N
  PK_PROJ_DOT,      // projection + <p, Ap>
  PK_UPDATE,        // x, r update + <r, r>
  PK_PROJECT,       // projection alone
  PK_RESIDUAL,      // FP64 residual b - G A x
  PK_GRAM_ROW,      // last-axis inverse + Gram sums
  PK_MISC,          // conversions, init, right-hand side
  PK_COUNT
};

int prof_begin(ghb_ctx* c, int pk, bool f32) {
  if (!c->prof) return -1;
  const int n = c->nrec;
  while (static_cast<int>(c->ev.size()) < 2 * (n + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->ev.push_back(e);
  }
  if (static_cast<int>(c->rec_cls.size()) < n + 1) c->rec_cls.resize(n + 1);
  c->rec_cls[n] = 2 * pk + (f32 ? 1 : 0);
  cudaEventRecord(c->ev[2 * n], c->stream);
  return n;
}

void prof_end(ghb_ctx* c, int n) {
  if (n < 0) return;
  cudaEventRecord(c->ev[2 * n + 1], c->stream);
  c->nrec = n + 1;
}

#define PROF(c, pk, f32, expr)                 \
  do {                                         \
    const int pn__ = prof_begin((c), (pk), (f32)); \
    ghb_status ps__ = (expr);                  \
    prof_end((c), pn__);                       \
    if (ps__ != GHB_OK) return ps__;           \
  } while (0)

double periodic_gap(double a, double b) {
  double t = a - b;
  t -= std::nearbyint(t);
  return std::fabs(t);
}

// Non-overlap of two inclusions in the periodic cell (touching is allowed).
bool overlap(int d, const ghb_phase& p, const ghb_phase& q) {
  const bool pr = p.shape != GHB_BOX, qr = q.shape != GHB_BOX;
  if (!pr && !qr) {
    for (int a = 0; a < d; ++a)
      if (periodic_gap(p.center[a], q.center[a]) >= 0.5 * (p.size[a] + q.size[a])) return false;
    return true;
  }
  if (pr && qr) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
      const double t = periodic_gap(p.center[a], q.center[a]);
      s += t * t;
    }
    return std::sqrt(s) < p.size[0] + q.size[0];
  }
  const ghb_phase& box = pr ? q : p;
  const ghb_phase& ball = pr ? p : q;
  double s = 0.0;
  for (int a = 0; a < d; ++a) {
    double t = periodic_gap(ball.center[a], box.center[a]) - 0.5 * box.size[a];
    if (t > 0) s += t * t;
  }
  return std::sqrt(s) < ball.size[0];
}

ghb_status validate_phases(int d, double a0, const ghb_phase* phases, int n) {
  if (!(a0 > 0.0) || !std::isfinite(a0)) {
    set_error("matrix coefficient a0 must be positive and finite (eq. A)");
    return GHB_ERR_INVALID;
  }
  if (n < 0 || (n > 0 && phases == nullptr)) {
    set_error("phases: null pointer or negative count");
    return GHB_ERR_INVALID;
  }
  for (int i = 0; i < n; ++i) {
    const ghb_phase& p = phases[i];
    if (!(p.value > 0.0) || !std::isfinite(p.value)) {
      set_error("inclusion " + std::to_string(i) + ": coefficient must be positive and finite");
      return GHB_ERR_INVALID;
    }
    for (int a = 0; a < d; ++a)
      if (!std::isfinite(p.center[a])) {
        set_error("inclusion " + std::to_string(i) + ": non-finite centre");
        return GHB_ERR_INVALID;
      }
    if (p.shape == GHB_BOX) {
      for (int a = 0; a < d; ++a)
        if (!(p.size[a] > 0.0 && p.size[a] <= 1.0)) {
          set_error("inclusion " + std::to_string(i) + ": box sides must lie in (0, 1]");
          return GHB_ERR_INVALID;
        }
    } else if ((p.shape == GHB_DISK && d == 2) || (p.shape == GHB_SPHERE && d == 3)) {
      if (!(p.size[0] > 0.0 && p.size[0] <= 0.5)) {
        set_error("inclusion " + std::to_string(i) + ": radius must lie in (0, 1/2]");
        return GHB_ERR_INVALID;
      }
    } else {
      set_error("inclusion " + std::to_string(i) + ": shape not valid in this dimension");
      return GHB_ERR_INVALID;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (overlap(d, phases[i], phases[j])) {
        set_error("inclusions " + std::to_string(i) + " and " + std::to_string(j) +
                  " overlap (the table of 1/a needs disjoint inclusions)");
        return GHB_ERR_INVALID;
      }
  return GHB_OK;
}

// a^ (kind 0, values a) or (1/a)^ (kind 1, values 1/a) on Z_{2N-1}, then the
// double-grid values (eq. MBA_GA) by the same padded inverse transforms as a
// field (Remark eval_with_FFT).
// Double-grid values A_M (eq. MBA_GA) of the table c->tab[kind]: the inverse
// transforms of the table zero-padded from Z_{2N-1} to the double grid, then
// the FP32 copy of the inner CG.
ghb_status grids_from_table(ghb_ctx* c, int kind) {
  const Geometry& g = c->g;
    const int Nd = g.N[g.d - 1];
    if (g.d == 2) {
      ColArgs a{};
      a.in = c->tab[kind];
      a.out = c->tabT1;
      a.outer = 1;
      a.inner = Nd;
      a.Lin = 2 * g.N[0] - 1;
      a.Lout = g.M[0];
      PROF(c, PK_COEFF, false, launch_col<double>(+1, COL_PLAIN, a, plan_of(c, 0), c->stream));
      RowArgs r{};
      r.t[0] = c->tabT1;
      r.nfields = 1;
      r.ncomp = 1;
      r.rows = g.M[0];
      r.H = Nd;
      r.comp_stride = 0;
      r.out_real = c->grid64[kind];
      PROF(c, PK_COEFF, false, launch_row<double>(ROW_TOREAL, r, plan_of(c, 1), c->stream));
    } else {
      ColArgs a{};
      a.in = c->tab[kind];
      a.out = c->tabT1;
      a.outer = 1;
      a.inner = static_cast<int64_t>(2 * g.N[1] - 1) * Nd;
      a.Lin = 2 * g.N[0] - 1;
      a.Lout = g.M[0];
      PROF(c, PK_COEFF, false, launch_col<double>(+1, COL_PLAIN, a, plan_of(c, 0), c->stream));
      ColArgs b{};
      b.in = c->tabT1;
      b.out = c->tabT2;
      b.outer = g.M[0];
      b.inner = Nd;
      b.Lin = 2 * g.N[1] - 1;
      b.Lout = g.M[1];
      PROF(c, PK_COEFF, false, launch_col<double>(+1, COL_PLAIN, b, plan_of(c, 1), c->stream));
      RowArgs r{};
      r.t[0] = c->tabT2;
      r.nfields = 1;
      r.ncomp = 1;
      r.rows = static_cast<int64_t>(g.M[0]) * g.M[1];
      r.H = Nd;
      r.out_real = c->grid64[kind];
      PROF(c, PK_COEFF, false, launch_row<double>(ROW_TOREAL, r, plan_of(c, 2), c->stream));
    }
    PROF(c, PK_COEFF, false, launch_to_f32_real(c->grid32[kind], c->grid64[kind], g.grid, c->stream));
  return GHB_OK;
}

ghb_status build_coeffs(ghb_ctx* c, double a0, const ghb_phase* phases, int n) {
  const Geometry& g = c->g;
  c->a0 = a0;
  c->n_incs = n;
  c->is_image = false;
  c->red_ready = false;
  c->gani_ready = false;   // the GaNi samples follow the new microstructure on next use
  if (n > c->incs_cap) {   // two lists: kind 0 (a) and kind 1 (1/a)
    if (c->d_incs) cudaFree(c->d_incs);
    c->d_incs = nullptr;
    c->incs_cap = 0;
    TRY(dmalloc(c, &c->d_incs, 2 * static_cast<int64_t>(n)));
    c->incs_cap = n;
  }
  for (int kind = 0; kind < 2; ++kind) {
    std::vector<Incl> h(n);
    const double a0v = kind == 0 ? a0 : 1.0 / a0;
    for (int i = 0; i < n; ++i) {
      Incl& in = h[i];
      in.shape = phases[i].shape;
      in.pad = 0;
      for (int a = 0; a < 3; ++a) {
        in.c[a] = a < g.d ? phases[i].center[a] : 0.0;
        in.s[a] = phases[i].size[a];
      }
      const double v = kind == 0 ? phases[i].value : 1.0 / phases[i].value;
      in.dv = v - a0v;
      in.v = v;
    }
    if (n > 0) {
      GHB_CUDA_TRY(cudaMemcpy(c->d_incs + kind * c->incs_cap, h.data(), sizeof(Incl) * n,
                              cudaMemcpyHostToDevice));
    }
  }
  // both tables in one pass (shared shape factors and phases)
  PROF(c, PK_COEFF, false,
       launch_coeff_tables(c->tab[0], c->tab[1], g, c->d_incs, c->d_incs + c->incs_cap, n, a0, 1.0 / a0,
                           c->stream));
  for (int kind = 0; kind < 2; ++kind) TRY(grids_from_table(c, kind));
  return GHB_OK;
}

// Coefficient tables of a piecewise-constant pixel image (Lemma grid_compos,
// Remark eval_with_FFT): the normalised P-sized DFT of the image (kind 0) and
// of its inverse (kind 1) through the column passes, one axis at a time, then
// a^(m) = prod_a sinc(m_a / P_a) C^(m mod P) on Z_{2N-1}, then the grid values.
ghb_status build_image(ghb_ctx* c, const int* P, const double* image) {
  const Geometry& g = c->g;
  const int d = g.d;
  int64_t np = 1;
  for (int a = 0; a < d; ++a) np *= P[a];
  c->is_image = true;
  c->red_ready = false;
  c->gani_ready = false;
  std::vector<double2> h(np);
  struct Scratch {   // two image-sized buffers, released on every exit
    double2* p[2] = {nullptr, nullptr};
    ~Scratch() {
      for (double2* q : p)
        if (q) cudaFree(q);
    }
  } sc;
  GHB_CUDA_TRY(cudaMalloc(&sc.p[0], sizeof(double2) * np));
  GHB_CUDA_TRY(cudaMalloc(&sc.p[1], sizeof(double2) * np));
  double2* A = sc.p[0];
  double2* B = sc.p[1];
  PlanHolder plans[3];
  struct FreePlans {
    PlanHolder* p;
    ~FreePlans() {
      for (int a = 0; a < 3; ++a) free_plan(p[a]);
    }
  } fp{plans};
  for (int a = 0; a < d; ++a) TRY(make_plan_untuned(P[a], plans[a]));
  int Pc[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) Pc[a] = P[a];
  for (int kind = 0; kind < 2; ++kind) {
    for (int64_t i = 0; i < np; ++i) h[i] = make_double2(kind == 0 ? image[i] : 1.0 / image[i], 0.0);
    GHB_CUDA_TRY(cudaMemcpyAsync(A, h.data(), sizeof(double2) * np, cudaMemcpyHostToDevice, c->stream));
    double2* src = A;
    double2* dst = B;
    int64_t outer = 1;
    for (int a = 0; a < d; ++a) {
      int64_t inner = 1;
      for (int b2 = a + 1; b2 < d; ++b2) inner *= P[b2];
      ColArgs f{};
      f.in = src;
      f.out = dst;
      f.outer = outer;
      f.inner = inner;
      f.Lin = P[a];
      f.Lout = P[a];
      PROF(c, PK_COEFF, false, launch_col<double>(-1, COL_PLAIN, f, plans[a].plan, c->stream));
      std::swap(src, dst);
      outer *= P[a];
    }
    PROF(c, PK_COEFF, false, launch_image_table(c->tab[kind], g, src, Pc, c->stream));
    TRY(grids_from_table(c, kind));
  }
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));   // before the scratch is released
  return GHB_OK;
}

// The passes of one operator application A^full x -> w (not yet projected)
// through the active view c->op, reading x from `in` (the first column pass
// may also form p = r + beta p_old).
template <typename C>
ghb_status operator_passes_view(ghb_ctx* c, int kind, const C* in, C* out, C* T1, C* T2, const CgState* st,
                                bool pupdate, const C* pold, C* pnew) {
  using T = decltype(C{}.x);
  const OpView& V = *c->op;
  const Geometry& g = V.g;
  const int d = g.d;
  const void* grid = (sizeof(T) == 8) ? static_cast<const void*>(V.grid64[kind])
                                      : static_cast<const void*>(V.grid32[kind]);
  ColArgs a{};
  a.in = in;
  a.out = T1;
  a.pold = pold;
  a.pnew = pnew;
  a.st = st;
  a.outer = d;
  a.inner = g.P / g.N[0];
  a.Lin = g.N[0];
  a.Lout = g.M[0];
  constexpr bool f32 = sizeof(T) == 4;
  PROF(c, pupdate ? PK_COL1_INV_PU : PK_COL1_INV, f32,
       launch_col<T>(+1, pupdate ? COL_PUPDATE : COL_PLAIN, a, *V.plan[0], c->stream));
  C* last = T1;
  if (d == 3) {
    ColArgs b{};
    b.in = T1;
    b.out = T2;
    b.st = st;
    b.outer = static_cast<int64_t>(d) * g.M[0];
    b.inner = g.h;
    b.Lin = g.N[1];
    b.Lout = g.M[1];
    PROF(c, PK_COL2_INV, f32, launch_col<T>(+1, COL_PLAIN, b, *V.plan[1], c->stream));
    last = T2;
  }
  RowArgs r{};
  r.t[0] = last;
  r.nfields = 1;
  r.ncomp = d;
  r.rows = g.rows;
  r.H = g.h;
  r.comp_stride = g.rows * g.h;
  r.a = grid;
  r.st = st;
  PROF(c, PK_ROW, f32, launch_row<T>(ROW_MATVEC, r, *V.plan[d - 1], c->stream));
  if (d == 3) {
    ColArgs b{};
    b.in = T2;
    b.out = T1;
    b.st = st;
    b.outer = static_cast<int64_t>(d) * g.M[0];
    b.inner = g.h;
    b.Lin = g.M[1];
    b.Lout = g.N[1];
    PROF(c, PK_COL2_FWD, f32, launch_col<T>(-1, COL_PLAIN, b, *V.plan[1], c->stream));
  }
  ColArgs f{};
  f.in = T1;
  f.out = out;
  f.st = st;
  f.outer = d;
  f.inner = g.P / g.N[0];
  f.Lin = g.M[0];
  f.Lout = g.N[0];
  PROF(c, PK_COL1_FWD, f32, launch_col<T>(-1, COL_PLAIN, f, *V.plan[0], c->stream));
  return GHB_OK;
}

template <typename C>
Work<C>& work(ghb_ctx* c);
template <>
Work<double2>& work<double2>(ghb_ctx* c) { return c->w64; }
template <>
Work<float2>& work<float2>(ghb_ctx* c) { return c->w32; }

ghb_status ensure_reduced(ghb_ctx* c);

// One operator application A^full x -> w: the active view's passes, or for the
// Ga operator in its reduced form (Lemma reduce_grid, Algorithm 3)
//   w = 2^-d sum_s S*(s) F_N [A_N(s) . F_N^-1 S(s) x],  S(s) = diag(omega_2N^{-s.m}),
// each shift through the N-grid passes with the double-grid values at 2r - s
// (the shift s = 0 carries the fused p update).
template <typename C>
ghb_status operator_passes(ghb_ctx* c, int kind, const C* in, C* out, C* T1, C* T2, const CgState* st,
                           bool pupdate, const C* pold, C* pnew) {
  if (c->op != &c->ga || c->form != GHB_FORM_REDUCED)
    return operator_passes_view<C>(c, kind, in, out, T1, T2, st, pupdate, pold, pnew);
  using T = decltype(C{}.x);
  if (!c->red_ready) TRY(ensure_reduced(c));
  Work<C>& W = work<C>(c);
  const FieldGeom fg = fgeom(c->g);
  const int ns = 1 << c->g.d;
  const double sc = 1.0 / ns;
  constexpr bool f32 = sizeof(T) == 4;
  const OpView* saved = c->op;
  c->op = &c->red[0];
  ghb_status st0 = operator_passes_view<C>(c, kind, in, out, T1, T2, st, pupdate, pold, pnew);
  const C* x = pupdate ? pnew : in;
  for (int sh = 1; sh < ns && st0 == GHB_OK; ++sh) {
    PROF(c, PK_MISC, f32, launch_phase<T>(W.s1, x, fg, sh, -1, 0.0, 1.0, st, c->stream));
    c->op = &c->red[sh];
    st0 = operator_passes_view<C>(c, kind, W.s1, W.s2, T1, T2, st, false, nullptr, nullptr);
    if (st0 != GHB_OK) break;
    const bool last = sh == ns - 1;
    PROF(c, PK_MISC, f32, launch_phase<T>(out, W.s2, fg, sh, +1, last ? sc : 1.0, last ? sc : 1.0, st,
                                          c->stream));
  }
  c->op = saved;
  return st0;
}

// One CG iteration (Remark CG) on the work buffers of precision C; every
// kernel returns at once when the device state says the solve is over.
template <typename C>
ghb_status cg_iteration(ghb_ctx* c, int kind) {
  using T = decltype(C{}.x);
  Work<C>& W = work<C>(c);
  const FieldGeom fg = fgeom(c->g);
  TRY(operator_passes<C>(c, kind, W.r, W.w, W.T1, W.T2, c->st, true, W.p, W.p));
  constexpr bool f32 = sizeof(T) == 4;
  PROF(c, PK_PROJ_DOT, f32, launch_project_dot<T>(W.q, W.w, W.p, fg, kind, c->st, c->partials, c->stream));
  PROF(c, PK_UPDATE, f32, launch_update<T>(W.x, W.r, W.p, W.q, fg, c->st, c->partials, c->stream));
  return GHB_OK;
}

ghb_status read_state(ghb_ctx* c) {
  GHB_CUDA_TRY(cudaMemcpyAsync(c->h_st, c->st, sizeof(CgState), cudaMemcpyDeviceToHost, c->stream));
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return GHB_OK;
}

// CG on W.{x,r,p} with the right-hand side already in W.r... initialised by
// cg_init; runs until the device state reports the end.
template <typename C>
ghb_status cg_run(ghb_ctx* c, int kind, const C* b, double tol, int maxiter, int* iters_out,
                  int* done_out, double* rr_out, double* bb_out) {
  using T = decltype(C{}.x);
  Work<C>& W = work<C>(c);
  const FieldGeom fg = fgeom(c->g);
  PROF(c, PK_MISC, sizeof(T) == 4, launch_cg_init<T>(W.x, W.r, W.p, b, fg, c->st, c->partials, tol, maxiter, c->stream));
  TRY(read_state(c));
  int chunk = 4;
  int mark[32];
  while (c->h_st->done == RUNNING) {
    const int base = c->h_st->iter;
    for (int i = 0; i < chunk; ++i) {
      mark[i] = c->nrec;
      TRY(cg_iteration<C>(c, kind));
    }
    TRY(read_state(c));
    // launches queued after the solve ended returned at once: drop their timings
    const int ran = c->h_st->iter - base;
    if (c->prof && c->h_st->done != RUNNING && ran >= 0 && ran < chunk) c->nrec = mark[ran];
    if (chunk < 32) chunk *= 2;
  }
  *iters_out = c->h_st->iter;
  *done_out = c->h_st->done;
  *rr_out = c->h_st->rr;
  *bb_out = c->h_st->bb;
  return GHB_OK;
}

// y = G A x (project) or A x, FP64 or FP32, through the context's work buffers.
template <typename C>
ghb_status apply_op(ghb_ctx* c, int kind, const C* x, C* y, bool project) {
  using T = decltype(C{}.x);
  Work<C>& W = work<C>(c);
  TRY(operator_passes<C>(c, kind, x, project ? W.w : y, W.T1, W.T2, nullptr, false, nullptr,
                         nullptr));
  if (project) PROF(c, PK_PROJECT, sizeof(T) == 4, launch_project<T>(y, W.w, fgeom(c->g), kind, c->stream));
  return GHB_OK;
}

// Gram matrix (1/|M|) sum_m A_M(x_m) v_i(x_m).v_j(x_m) of m FP64 fields
// (Lemma integ_eval_VM): inverse passes of each field, then one Gram pass.
ghb_status gram(ghb_ctx* c, const OpView& V, int kind, int m, const double2* const* fields, double* out) {
  const Geometry& g = V.g;
  const int d = g.d;
  RowArgs r{};
  for (int f = 0; f < m; ++f) {
    ColArgs a{};
    a.in = fields[f];
    a.out = c->gT1[f];
    a.outer = d;
    a.inner = g.P / g.N[0];
    a.Lin = g.N[0];
    a.Lout = g.M[0];
    PROF(c, PK_COL1_INV, false, launch_col<double>(+1, COL_PLAIN, a, *V.plan[0], c->stream));
    r.t[f] = c->gT1[f];
    if (d == 3) {
      ColArgs b{};
      b.in = c->gT1[f];
      b.out = c->gT2[f];
      b.outer = static_cast<int64_t>(d) * g.M[0];
      b.inner = g.h;
      b.Lin = g.N[1];
      b.Lout = g.M[1];
      PROF(c, PK_COL2_INV, false, launch_col<double>(+1, COL_PLAIN, b, *V.plan[1], c->stream));
      r.t[f] = c->gT2[f];
    }
  }
  r.nfields = m;
  r.ncomp = d;
  r.rows = g.rows;
  r.H = g.h;
  r.comp_stride = g.rows * g.h;
  r.a = V.grid64[kind];
  r.partials = c->partials;
  r.gram = c->d_gram;
  r.ticket = c->ticket;
  r.scale = 1.0 / static_cast<double>(g.grid);
  PROF(c, PK_GRAM_ROW, false, launch_row<double>(ROW_ENERGY, r, *V.plan[d - 1], c->stream));
  GHB_CUDA_TRY(cudaMemcpyAsync(c->h_gram, c->d_gram, sizeof(double) * m * m, cudaMemcpyDeviceToHost,
                               c->stream));
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < m * m; ++i) out[i] = c->h_gram[i];
  return GHB_OK;
}

// One solve: minimiser over E_N (primal) / J_N (dual) for load E; the
// admissible field E + e (FP64) is left in `field_out` (device).
// Exact energy a(E + e, E + e) (or a^{-1}) of the admissible field E + e held in
// `scratch` after the call (Gram on the double grid).
ghb_status energy_of(ghb_ctx* c, int kind, const double* E, const double2* e, double2* scratch, double* out) {
  PROF(c, PK_MISC, false, launch_add_constant(scratch, e, fgeom(c->g), E, c->stream));
  const double2* f = scratch;
  return gram(c, c->ga, kind, 1, &f, out);
}

// Sets (or clears, hist = nullptr) the bound-tracking buffer of the CG state.
ghb_status set_history(ghb_ctx* c, double* hist, int cap) {
  CgState h{};
  h.hist = hist;
  h.hist_cap = cap;
  GHB_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(c->st) + offsetof(CgState, hist), &h.hist,
                               sizeof(double*) + sizeof(int), cudaMemcpyHostToDevice, c->stream));
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return GHB_OK;
}

// One solve: minimiser over E_N (primal) / J_N (dual) for load E; the
// admissible field E + e (FP64) is left in `field_out` (device).  x0: initial
// fluctuation (admissible, FP64; null = 0).  energies: if not null, receives the
// energy of E + e along the iterates (bound tracking, Section 7.4): FP64, every
// CG iterate, J(x_i) = J(x_0) - sum_{j<i} alpha_j <r_j, r_j>; mixed, the start
// and every FP64 correction, each an exact Gram evaluation.
// With ax_out (mixed precision only), the operator output of the returned
// iterate before projection -- left in the FP64 work buffer by the last
// residual correction -- is copied there and *ax_ok says whether it was.
ghb_status solve(ghb_ctx* c, int kind, const double* E, double2* field_out, ghb_solve_info* info,
                 const double2* x0 = nullptr, std::vector<double>* energies = nullptr,
                 double2* ax_out = nullptr, bool* ax_ok = nullptr) {
  if (ax_ok) *ax_ok = false;
  const Geometry& g = c->g;
  const FieldGeom fg = fgeom(g);
  ghb_solve_info inf{};
  if (c->op == &c->gani) {
    // b = -G (a~ E)^: the constant field E through the unprojected operator
    GHB_CUDA_TRY(cudaMemsetAsync(c->b64, 0, sizeof(double2) * g.field, c->stream));
    PROF(c, PK_MISC, false, launch_add_constant(c->y64, c->b64, fg, E, c->stream));
    TRY(apply_op<double2>(c, kind, c->y64, c->b64, true));
    PROF(c, PK_MISC, false, launch_scale(c->b64, -1.0, g.field, c->stream));
  } else {
    PROF(c, PK_MISC, false, launch_rhs<double>(c->b64, c->tab[kind], g, E, kind, c->stream));
  }
  const double tol = c->opt.tol;
  const int maxiter = c->opt.max_iter;
  int iters = 0, done = RUNNING;
  double rr = 0, bb = 0;
  double J0 = 0.0;
  if (energies) {
    energies->clear();
    if (x0) {
      TRY(energy_of(c, kind, E, x0, field_out, &J0));
    } else {
      GHB_CUDA_TRY(cudaMemsetAsync(c->w64.q, 0, sizeof(double2) * g.field, c->stream));
      TRY(energy_of(c, kind, E, c->w64.q, field_out, &J0));
    }
  }
  if (c->opt.precision == GHB_FP64) {
    const double2* rhs = c->b64;
    double tol_run = tol, bb_full = 0.0;
    if (x0) {
      // ||b||^2, then b' = b - G A x0 (x0 admissible); CG on the correction
      GHB_CUDA_TRY(cudaMemsetAsync(c->w64.q, 0, sizeof(double2) * g.field, c->stream));
      PROF(c, PK_RESIDUAL, false, launch_residual(c->y64, c->b64, c->w64.q, fg, c->st, c->partials, c->stream));
      TRY(read_state(c));
      bb_full = c->h_st->rr;
      TRY(apply_op<double2>(c, kind, x0, c->w64.q, true));
      PROF(c, PK_RESIDUAL, false, launch_residual(c->y64, c->b64, c->w64.q, fg, c->st, c->partials, c->stream));
      TRY(read_state(c));
      const double bbp = c->h_st->rr;
      rhs = c->y64;
      tol_run = bbp > 0 ? std::min(0.5, tol * std::sqrt(bb_full / bbp)) : tol;
    }
    if (energies) {
      const int cap = std::min(maxiter + 1, 1 << 20);
      if (c->hist_cap < cap) {
        if (c->d_hist) cudaFree(c->d_hist);
        c->d_hist = nullptr;
        c->hist_cap = 0;
        TRY(dmalloc(c, &c->d_hist, cap));
        c->hist_cap = cap;
      }
      TRY(set_history(c, c->d_hist, c->hist_cap));
    }
    const ghb_status st = cg_run<double2>(c, kind, rhs, tol_run, maxiter, &iters, &done, &rr, &bb);
    if (energies) TRY(set_history(c, nullptr, 0));
    TRY(st);
    if (x0) {
      PROF(c, PK_MISC, false, launch_axpy(c->w64.x, x0, 1.0, g.field, c->stream));
      bb = bb_full;
    }
    inf.iters = iters;
    inf.matvecs_fp64 = iters + (x0 ? 1 : 0);
    inf.relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    if (energies) {
      const int n = std::min(iters + 1, c->hist_cap);
      std::vector<double> h(n);
      GHB_CUDA_TRY(cudaMemcpyAsync(h.data(), c->d_hist, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
      GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
      for (int i = 0; i < n; ++i) energies->push_back(J0 - h[i]);
    }
    // exact projection of the iterate (admissibility up to FP64 rounding)
    PROF(c, PK_PROJECT, false, launch_project<double>(c->w64.q, c->w64.x, fg, kind, c->stream));
    PROF(c, PK_MISC, false, launch_add_constant(field_out, c->w64.q, fg, E, c->stream));
  } else {
    // FP64 residual correction around FP32 CG solves.  x64 (= y64) holds the
    // projected iterate, w64.x its unprojected accumulation.
    double2* x64 = c->y64;
    double2* r64 = c->w64.r;
    bool ax_valid = false;   // w64.w holds the unprojected operator output of x64
    // ||b||^2 through the FP64 residual kernel with y = 0
    GHB_CUDA_TRY(cudaMemsetAsync(c->w64.q, 0, sizeof(double2) * g.field, c->stream));
    PROF(c, PK_RESIDUAL, false, launch_residual(r64, c->b64, c->w64.q, fg, c->st, c->partials, c->stream));
    TRY(read_state(c));
    bb = c->h_st->rr;
    rr = bb;
    if (x0) {
      GHB_CUDA_TRY(cudaMemcpyAsync(x64, x0, sizeof(double2) * g.field, cudaMemcpyDeviceToDevice, c->stream));
      GHB_CUDA_TRY(cudaMemcpyAsync(c->w64.x, x0, sizeof(double2) * g.field, cudaMemcpyDeviceToDevice,
                                   c->stream));
      TRY(apply_op<double2>(c, kind, x64, c->w64.q, true));
      ax_valid = true;
      PROF(c, PK_RESIDUAL, false, launch_residual(r64, c->b64, c->w64.q, fg, c->st, c->partials, c->stream));
      TRY(read_state(c));
      rr = c->h_st->rr;
    } else {
      GHB_CUDA_TRY(cudaMemsetAsync(x64, 0, sizeof(double2) * g.field, c->stream));
      GHB_CUDA_TRY(cudaMemsetAsync(c->w64.x, 0, sizeof(double2) * g.field, c->stream));
    }
    if (energies) energies->push_back(J0);
    int outer = 0;
    int total_inner = 0, mv32 = 0, mv64 = 0;
    done = CONVERGED;
    while (bb > 0 && rr > tol * tol * bb) {
      if (outer >= c->opt.max_outer || total_inner >= maxiter) {
        done = MAXITER;
        break;
      }
      PROF(c, PK_MISC, true, launch_to_f32(c->w32.w, r64, fg, c->stream));
      // q32 holds the FP32 right-hand side for the inner solve
      GHB_CUDA_TRY(cudaMemcpyAsync(c->w32.q, c->w32.w, sizeof(float2) * g.field,
                                   cudaMemcpyDeviceToDevice, c->stream));
      int it = 0, dn = 0;
      double rr32 = 0, bb32 = 0;
      const double itol = inner_target(c->opt.inner_tol, tol, rr, bb);
      TRY(cg_run<float2>(c, kind, c->w32.q, itol, maxiter - total_inner, &it, &dn, &rr32, &bb32));
      total_inner += it;
      mv32 += it;
      if (dn == BREAKDOWN && it == 0) {
        done = BREAKDOWN;
        break;
      }
      PROF(c, PK_MISC, false, launch_accum_f32(c->w64.x, c->w64.x, c->w32.x, fg, c->stream));
      ax_valid = false;
      // exact FP64 projection onto the admissible (real, curl- or divergence-free) fields
      PROF(c, PK_PROJECT, false, launch_project<double>(x64, c->w64.x, fg, kind, c->stream));
      GHB_CUDA_TRY(cudaMemcpyAsync(c->w64.x, x64, sizeof(double2) * g.field, cudaMemcpyDeviceToDevice,
                                   c->stream));
      TRY(apply_op<double2>(c, kind, x64, c->w64.q, true));
      ax_valid = true;
      mv64 += 1;
      PROF(c, PK_RESIDUAL, false, launch_residual(r64, c->b64, c->w64.q, fg, c->st, c->partials, c->stream));
      TRY(read_state(c));
      rr = c->h_st->rr;
      ++outer;
      if (!std::isfinite(rr)) {
        done = BREAKDOWN;
        break;
      }
      if (energies) {
        double J = 0.0;
        TRY(energy_of(c, kind, E, x64, field_out, &J));
        energies->push_back(J);
        ax_valid = false;
      }
    }
    if (ax_out && ax_valid) {
      GHB_CUDA_TRY(cudaMemcpyAsync(ax_out, c->w64.w, sizeof(double2) * g.field, cudaMemcpyDeviceToDevice,
                                   c->stream));
      if (ax_ok) *ax_ok = true;
    }
    inf.iters = total_inner;
    inf.outer_iters = outer;
    inf.matvecs_fp32 = mv32;
    inf.matvecs_fp64 = mv64;
    inf.relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    PROF(c, PK_MISC, false, launch_add_constant(field_out, x64, fg, E, c->stream));
  }
  inf.status = done == CONVERGED ? GHB_OK : (done == BREAKDOWN ? GHB_ERR_BREAKDOWN : GHB_ERR_NOT_CONVERGED);
  if (info) *info = inf;
  return GHB_OK;
}

void free_ctx(ghb_ctx* c) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  for (auto& p : c->plan) free_plan(p);
  for (auto& p : c->planN) free_plan(p);
  for (int k = 0; k < 2; ++k) {
    F(c->redgrid64[k]);
    F(c->redgrid32[k]);
    F(c->gridN64[k]);
    F(c->gridN32[k]);
    F(c->tab[k]);
    F(c->grid64[k]);
    F(c->grid32[k]);
  }
  F(c->tabT1);
  F(c->tabT2);
  F(c->d_hist);
  F(c->d_incs);
  for (auto* W : {&c->w64}) {
    F(W->x); F(W->r); F(W->p); F(W->q); F(W->w); F(W->T1); F(W->T2); F(W->s1); F(W->s2);
  }
  for (auto* W : {&c->w32}) {
    F(W->x); F(W->r); F(W->p); F(W->q); F(W->w); F(W->T1); F(W->T2); F(W->s1); F(W->s2);
  }
  F(c->b64);
  F(c->y64);
  for (int i = 0; i < 3; ++i) {
    F(c->sol[i]);
    F(c->gT1[i]);
    F(c->gT2[i]);
  }
  F(c->st);
  F(c->partials);
  F(c->ticket);
  F(c->d_gram);
  if (c->h_st) cudaFreeHost(c->h_st);
  if (c->h_gram) cudaFreeHost(c->h_gram);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

ghb_status alloc_ctx(ghb_ctx* c) {
  const Geometry& g = c->g;
  const int d = g.d;
  // plans: one per distinct M
  for (int a = 0; a < d; ++a) {
    int found = -1;
    for (int b = 0; b < a; ++b)
      if (g.M[b] == g.M[a]) found = c->plan_of_axis[b];
    if (found >= 0) {
      c->plan_of_axis[a] = found;
    } else {
      c->plan_of_axis[a] = a;
      TRY(make_plan(g.M[a], c->plan[a]));
    }
  }
  int64_t t1tab, t2tab = 0;
  if (d == 2) {
    t1tab = static_cast<int64_t>(g.M[0]) * g.N[1];
  } else {
    t1tab = static_cast<int64_t>(g.M[0]) * (2 * g.N[1] - 1) * g.N[2];
    t2tab = static_cast<int64_t>(g.M[0]) * g.M[1] * g.N[2];
  }
  for (int k = 0; k < 2; ++k) {
    TRY(dmalloc(c, &c->tab[k], g.table));
    TRY(dmalloc(c, &c->grid64[k], g.grid));
    TRY(dmalloc(c, &c->grid32[k], g.grid));
  }
  TRY(dmalloc(c, &c->tabT1, t1tab));
  if (d == 3) TRY(dmalloc(c, &c->tabT2, t2tab));
  auto alloc_work = [&](auto& W) -> ghb_status {
    TRY(dmalloc(c, &W.x, g.field));
    TRY(dmalloc(c, &W.r, g.field));
    TRY(dmalloc(c, &W.p, g.field));
    TRY(dmalloc(c, &W.q, g.field));
    TRY(dmalloc(c, &W.w, g.field));
    TRY(dmalloc(c, &W.T1, g.T1));
    if (d == 3) TRY(dmalloc(c, &W.T2, g.T2));
    return GHB_OK;
  };
  TRY(alloc_work(c->w64));
  TRY(alloc_work(c->w32));
  TRY(dmalloc(c, &c->b64, g.field));
  TRY(dmalloc(c, &c->y64, g.field));
  for (int i = 0; i < d; ++i) {
    TRY(dmalloc(c, &c->sol[i], g.field));
    TRY(dmalloc(c, &c->gT1[i], g.T1));
    if (d == 3) TRY(dmalloc(c, &c->gT2[i], g.T2));
  }
  TRY(dmalloc(c, &c->st, 1));
  TRY(dmalloc(c, &c->partials, kMaxPartials * 6));
  TRY(dmalloc(c, &c->ticket, 1));
  TRY(dmalloc(c, &c->d_gram, 9));
  GHB_CUDA_TRY(cudaMemset(c->st, 0, sizeof(CgState)));
  GHB_CUDA_TRY(cudaMemset(c->ticket, 0, sizeof(unsigned int)));
  GHB_CUDA_TRY(cudaMallocHost(&c->h_st, sizeof(CgState)));
  GHB_CUDA_TRY(cudaMallocHost(&c->h_gram, sizeof(double) * 9));
  c->ga.g = g;
  for (int a = 0; a < d; ++a) c->ga.plan[a] = &c->plan[c->plan_of_axis[a]].plan;
  for (int k = 0; k < 2; ++k) {
    c->ga.grid64[k] = c->grid64[k];
    c->ga.grid32[k] = c->grid32[k];
  }
  c->op = &c->ga;
  return GHB_OK;
}

// Plans of length N_a (the N-grid operators: GaNi and the reduced Ga form).
ghb_status ensure_planN(ghb_ctx* c) {
  const Geometry& g = c->g;
  const int d = g.d;
  if (c->planN[c->planN_of_axis[0]].d_perm != nullptr) return GHB_OK;
  for (int a = 0; a < d; ++a)
    if (!factorizable(g.N[a])) {
      set_error("the N-grid transforms have length N; N=" + std::to_string(g.N[a]) +
                " has a prime factor above 31");
      return GHB_ERR_INVALID;
    }
  for (int a = 0; a < d; ++a) {
    int found = -1;
    for (int b = 0; b < a; ++b)
      if (g.N[b] == g.N[a]) found = c->planN_of_axis[b];
    if (found >= 0) {
      c->planN_of_axis[a] = found;
    } else {
      c->planN_of_axis[a] = a;
      TRY(make_plan(g.N[a], c->planN[a]));
    }
  }
  return GHB_OK;
}

// Geometry of the operators on the N grid (M = N).
Geometry n_geometry(const Geometry& g) {
  Geometry gn = g;
  const int d = g.d;
  for (int a = 0; a < d; ++a) gn.M[a] = g.N[a];
  gn.T1 = static_cast<int64_t>(d) * gn.M[0] * (g.P / g.N[0]);
  gn.T2 = d == 3 ? static_cast<int64_t>(d) * gn.M[0] * gn.M[1] * g.h : 0;
  gn.rows = d == 2 ? gn.M[0] : static_cast<int64_t>(gn.M[0]) * gn.M[1];
  gn.grid = 1;
  for (int a = 0; a < d; ++a) gn.grid *= gn.M[a];
  return gn;
}

// The reduced form (Lemma reduce_grid): for every shift s the N-grid view with
// the double-grid values at 2r - s; needs M = 2N on every axis.  Built on first
// use and refreshed after the coefficients change.
ghb_status ensure_reduced(ghb_ctx* c) {
  const Geometry& g = c->g;
  const int d = g.d;
  const int ns = 1 << d;
  if (c->red[0].plan[0] == nullptr) {
    for (int a = 0; a < d; ++a)
      if (g.M[a] != 2 * g.N[a]) {
        set_error("the reduced form needs the double grid M = 2N on every axis (Lemma reduce_grid)");
        return GHB_ERR_INVALID;
      }
    TRY(ensure_planN(c));
    const Geometry gn = n_geometry(g);
    for (int k = 0; k < 2; ++k) {
      TRY(dmalloc(c, &c->redgrid64[k], gn.grid * ns));
      TRY(dmalloc(c, &c->redgrid32[k], gn.grid * ns));
    }
    for (auto* W : {&c->w64}) {
      TRY(dmalloc(c, &W->s1, g.field));
      TRY(dmalloc(c, &W->s2, g.field));
    }
    for (auto* W : {&c->w32}) {
      TRY(dmalloc(c, &W->s1, g.field));
      TRY(dmalloc(c, &W->s2, g.field));
    }
    for (int sh = 0; sh < ns; ++sh) {
      c->red[sh].g = gn;
      for (int a = 0; a < d; ++a) c->red[sh].plan[a] = &c->planN[c->planN_of_axis[a]].plan;
      for (int k = 0; k < 2; ++k) {
        c->red[sh].grid64[k] = c->redgrid64[k] + sh * gn.grid;
        c->red[sh].grid32[k] = c->redgrid32[k] + sh * gn.grid;
      }
    }
  }
  if (!c->red_ready) {
    for (int k = 0; k < 2; ++k)
      for (int sh = 0; sh < ns; ++sh)
        PROF(c, PK_COEFF, false, launch_subgrid(c->red[sh].grid64[k], c->red[sh].grid32[k], c->grid64[k], g, sh,
                                                c->stream));
    c->red_ready = true;
  }
  return GHB_OK;
}

// The GaNi operator (Algorithm 1): transforms of length N (M = N), plans and
// the point samples of a and 1/a on the N grid; built on first use and
// resampled after ghb_set_coeffs.
ghb_status ensure_gani(ghb_ctx* c) {
  const Geometry& g = c->g;
  const int d = g.d;
  if (c->is_image) {
    set_error("the GaNi scheme is built for inclusion-matrix composites, not pixel images");
    return GHB_ERR_INVALID;
  }
  if (c->gani.plan[0] == nullptr) {
    TRY(ensure_planN(c));
    const Geometry gn = n_geometry(g);
    for (int k = 0; k < 2; ++k) {
      TRY(dmalloc(c, &c->gridN64[k], gn.grid));
      TRY(dmalloc(c, &c->gridN32[k], gn.grid));
    }
    c->gani.g = gn;
    for (int a = 0; a < d; ++a) c->gani.plan[a] = &c->planN[c->planN_of_axis[a]].plan;
    for (int k = 0; k < 2; ++k) {
      c->gani.grid64[k] = c->gridN64[k];
      c->gani.grid32[k] = c->gridN32[k];
    }
  }
  if (!c->gani_ready) {
    for (int kind = 0; kind < 2; ++kind)
      PROF(c, PK_COEFF, false, launch_sample_values(c->gridN64[kind], c->gridN32[kind], c->gani.g,
                                                    c->d_incs + kind * c->incs_cap, c->n_incs,
                                                    kind == 0 ? c->a0 : 1.0 / c->a0, c->stream));
    c->gani_ready = true;
  }
  return GHB_OK;
}

// Runs f with the GaNi operator active.
template <typename F>
ghb_status with_gani(ghb_ctx* c, F&& f) {
  TRY(ensure_gani(c));
  const OpView* saved = c->op;
  c->op = &c->gani;
  const ghb_status st = f();
  c->op = saved;
  return st;
}

// Inverse of a symmetric positive definite d x d matrix (d <= 3) by cofactors.
bool inverse_small(int d, const double* A, double* X) {
  if (d == 2) {
    const double det = A[0] * A[3] - A[1] * A[2];
    if (!(det > 0)) return false;
    X[0] = A[3] / det;
    X[1] = -A[1] / det;
    X[2] = -A[2] / det;
    X[3] = A[0] / det;
    return true;
  }
  const double c00 = A[4] * A[8] - A[5] * A[7];
  const double c01 = A[5] * A[6] - A[3] * A[8];
  const double c02 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  if (!(det > 0)) return false;
  X[0] = c00 / det;
  X[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  X[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  X[3] = c01 / det;
  X[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  X[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  X[6] = c02 / det;
  X[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  X[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return true;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
#define ABI_GUARD_BEGIN try {
#define ABI_GUARD_END                                   \
  }                                                     \
  catch (const std::exception& ex) {                    \
    set_error(std::string("internal error: ") + ex.what()); \
    return GHB_ERR_INVALID;                             \
  }

namespace {

ghb_status check_options(const ghb_options& o) {
  if (!(o.tol > 0.0 && o.tol < 1.0)) { set_error("options.tol must lie in (0, 1)"); return GHB_ERR_INVALID; }
  if (o.max_iter < 1) { set_error("options.max_iter must be >= 1"); return GHB_ERR_INVALID; }
  if (o.precision != GHB_FP64 && o.precision != GHB_MIXED) {
    set_error("options.precision must be GHB_FP64 or GHB_MIXED");
    return GHB_ERR_INVALID;
  }
  if (o.precision == GHB_MIXED && !(o.inner_tol > 0.0 && o.inner_tol < 1.0)) {
    set_error("options.inner_tol must lie in (0, 1)");
    return GHB_ERR_INVALID;
  }
  if (o.precision == GHB_MIXED && o.max_outer < 1) {
    set_error("options.max_outer must be >= 1");
    return GHB_ERR_INVALID;
  }
  return GHB_OK;
}

// The Gram pass holds up to 2 (d = 2) or 5 (d = 3) interleaved FP64 complex
// lines of length M in one CTA's shared memory (<= 200 KB).
constexpr int kMaxM2 = 6400;

// Algorithmic (compulsory) bytes and FFT flops of one launch of a kernel class.
// Bytes: each array the kernel must read or write, once.  Flops: 5 L log2 L per
// complex transform of length L (the usual FFT count), lines x transforms.
void algo_model(const ghb_ctx* c, int pk, bool f32, double* bytes, double* flops) {
  const Geometry& g = c->g;
  const double e = f32 ? 8.0 : 16.0, re = f32 ? 4.0 : 8.0;
  const double F = static_cast<double>(g.field);
  const double T1 = static_cast<double>(g.T1), T2 = static_cast<double>(g.T2);
  const double Tl = g.d == 3 ? T2 : T1;
  auto fft = [](double L) { return L > 1 ? 5.0 * L * std::log2(L) : 0.0; };
  const double M0 = g.M[0], M1 = g.M[1], Md = g.M[g.d - 1];
  const double lines1 = static_cast<double>(g.d) * (g.P / g.N[0]);   // axis-1 lines
  const double lines2 = static_cast<double>(g.d) * g.M[0] * g.h;    // axis-2 lines (d = 3)
  const double rowsc = static_cast<double>(g.rows) * g.d / 2.0;      // complex row transforms
  double b = 0, f = 0;
  switch (pk) {
    case PK_COL1_INV_PU: b = (3 * F + T1) * e; f = lines1 * fft(M0); break;
    case PK_COL1_INV: b = (F + T1) * e; f = lines1 * fft(M0); break;
    case PK_COL2_INV: b = (T1 + T2) * e; f = lines2 * fft(M1); break;
    case PK_ROW: b = 2 * Tl * e + static_cast<double>(g.grid) * re; f = rowsc * 2 * fft(Md); break;
    case PK_COL2_FWD: b = (T1 + T2) * e; f = lines2 * fft(M1); break;
    case PK_COL1_FWD: b = (T1 + F) * e; f = lines1 * fft(M0); break;
    case PK_PROJ_DOT: b = 3 * F * e; break;
    case PK_UPDATE: b = 6 * F * e; break;
    case PK_PROJECT: b = 2 * F * e; break;
    case PK_RESIDUAL: b = 3 * F * 16.0; break;
    case PK_GRAM_ROW:
      b = g.d * Tl * 16.0 + static_cast<double>(g.grid) * 8.0;
      f = static_cast<double>(g.rows) * g.d * g.d / 2.0 * fft(Md);
      break;
    default: break;
  }
  *bytes = b;
  *flops = f;
}
constexpr int kMaxM3 = 2560;

}  // namespace

extern "C" {

const char* ghb_version(void) { return "ghb 0.1 (sm_103a)"; }

const char* ghb_last_error(void) { return last_error_cstr(); }

void ghb_default_options(ghb_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->tol = 1e-10;
  opt->max_iter = 20000;
  opt->precision = GHB_FP64;
  opt->inner_tol = 1e-5;
  opt->max_outer = 20;
}

ghb_status ghb_create(ghb_ctx** out, int d, const int* N, double a0, const ghb_phase* phases,
                      int n_phases, const ghb_options* opt) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!out) { set_error("out is NULL"); return GHB_ERR_INVALID; }
  *out = nullptr;
  if (d != 2 && d != 3) { set_error("d must be 2 or 3"); return GHB_ERR_INVALID; }
  if (!N) { set_error("N is NULL"); return GHB_ERR_INVALID; }
  ghb_options o;
  ghb_default_options(&o);
  if (opt) o = *opt;
  TRY(check_options(o));
  Geometry g{};
  g.d = d;
  for (int a = 0; a < 3; ++a) { g.N[a] = 1; g.M[a] = 1; }
  for (int a = 0; a < d; ++a) {
    if (N[a] < 1 || N[a] % 2 == 0) {
      set_error("N must be odd and positive in every direction (eq. N_odd)");
      return GHB_ERR_INVALID;
    }
    g.N[a] = N[a];
    const int M = o.M[a] > 0 ? o.M[a] : auto_M(N[a]);
    if (M < 2 * N[a] - 1) {
      set_error("M must be >= 2N - 1 in every direction (Lemma integ_eval_VM)");
      return GHB_ERR_INVALID;
    }
    if (M > (d == 2 ? kMaxM2 : kMaxM3) || !factorizable(M)) {
      set_error("unsupported M=" + std::to_string(M) +
                " (prime factors <= 31; M <= 6400 for d = 2, M <= 2560 for d = 3)");
      return GHB_ERR_INVALID;
    }
    g.M[a] = M;
  }
  TRY(validate_phases(d, a0, phases, n_phases));
  g.h = (g.N[d - 1] + 1) / 2;
  g.P = g.h;
  for (int a = 0; a < d - 1; ++a) g.P *= g.N[a];
  g.field = static_cast<int64_t>(d) * g.P;
  g.T1 = static_cast<int64_t>(d) * g.M[0] * (g.P / g.N[0]);
  g.T2 = d == 3 ? static_cast<int64_t>(d) * g.M[0] * g.M[1] * g.h : 0;
  g.rows = d == 2 ? g.M[0] : static_cast<int64_t>(g.M[0]) * g.M[1];
  g.grid = 1;
  for (int a = 0; a < d; ++a) g.grid *= g.M[a];
  g.table = g.N[d - 1];
  for (int a = 0; a < d - 1; ++a) g.table *= (2 * g.N[a] - 1);

  ghb_ctx* c = new ghb_ctx();
  c->g = g;
  c->opt = o;
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    delete c;
    return GHB_ERR_CUDA;
  }
  c->stream = c->own_stream;
  ghb_status s = alloc_ctx(c);
  if (s == GHB_OK) s = build_coeffs(c, a0, phases, n_phases);
  if (s == GHB_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
    set_error(std::string("coefficient set-up: ") + cudaGetErrorString(cudaGetLastError()));
    s = GHB_ERR_CUDA;
  }
  if (s != GHB_OK) {
    free_ctx(c);
    return s;
  }
  *out = c;
  return GHB_OK;
  ABI_GUARD_END
}

ghb_status ghb_set_coeffs(ghb_ctx* c, double a0, const ghb_phase* phases, int n_phases) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c) { set_error("ctx is NULL"); return GHB_ERR_INVALID; }
  TRY(validate_phases(c->g.d, a0, phases, n_phases));
  TRY(build_coeffs(c, a0, phases, n_phases));
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return GHB_OK;
  ABI_GUARD_END
}

namespace {
ghb_status check_image(int d, const int* P, const double* image) {
  if (!P || !image) {
    set_error("P and image must not be NULL");
    return GHB_ERR_INVALID;
  }
  int64_t np = 1;
  for (int a = 0; a < d; ++a) {
    if (P[a] < 1 || P[a] > 8192 || !factorizable(P[a])) {
      set_error("image resolution P must lie in 1..8192 with prime factors <= 31");
      return GHB_ERR_INVALID;
    }
    np *= P[a];
  }
  for (int64_t i = 0; i < np; ++i)
    if (!(image[i] > 0.0) || !std::isfinite(image[i])) {
      set_error("image values must be positive and finite (eq. A)");
      return GHB_ERR_INVALID;
    }
  return GHB_OK;
}
}  // namespace

ghb_status ghb_create_image(ghb_ctx** out, int d, const int* N, const int* P, const double* image,
                            const ghb_options* opt) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!out) { set_error("out is NULL"); return GHB_ERR_INVALID; }
  *out = nullptr;
  if (d != 2 && d != 3) { set_error("d must be 2 or 3"); return GHB_ERR_INVALID; }
  TRY(check_image(d, P, image));
  ghb_ctx* c = nullptr;
  TRY(ghb_create(&c, d, N, 1.0, nullptr, 0, opt));
  const ghb_status s = build_image(c, P, image);
  if (s != GHB_OK) {
    ghb_destroy(c);
    return s;
  }
  *out = c;
  return GHB_OK;
  ABI_GUARD_END
}

ghb_status ghb_set_image(ghb_ctx* c, const int* P, const double* image) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c) { set_error("ctx is NULL"); return GHB_ERR_INVALID; }
  TRY(check_image(c->g.d, P, image));
  return build_image(c, P, image);
  ABI_GUARD_END
}

ghb_status ghb_set_form(ghb_ctx* c, int form) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c) { set_error("ctx is NULL"); return GHB_ERR_INVALID; }
  if (form != GHB_FORM_DOUBLE_GRID && form != GHB_FORM_REDUCED) {
    set_error("form must be GHB_FORM_DOUBLE_GRID or GHB_FORM_REDUCED");
    return GHB_ERR_INVALID;
  }
  if (form == GHB_FORM_REDUCED) {
    TRY(ensure_reduced(c));
    GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  c->form = form;
  return GHB_OK;
  ABI_GUARD_END
}

ghb_status ghb_set_options(ghb_ctx* c, const ghb_options* opt) {
  clear_error();
  if (!c || !opt) { set_error("ctx or opt is NULL"); return GHB_ERR_INVALID; }
  TRY(check_options(*opt));
  ghb_options o = *opt;
  for (int a = 0; a < 3; ++a) o.M[a] = c->opt.M[a];
  c->opt = o;
  return GHB_OK;
}

ghb_status ghb_set_stream(ghb_ctx* c, void* stream) {
  clear_error();
  if (!c) { set_error("ctx is NULL"); return GHB_ERR_INVALID; }
  c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
  return GHB_OK;
}

ghb_status ghb_get_grid(const ghb_ctx* c, int* d_out, int* N_out, int* M_out, int64_t* field_elems) {
  if (!c) { set_error("ctx is NULL"); return GHB_ERR_INVALID; }
  if (d_out) *d_out = c->g.d;
  for (int a = 0; a < c->g.d; ++a) {
    if (N_out) N_out[a] = c->g.N[a];
    if (M_out) M_out[a] = c->g.M[a];
  }
  if (field_elems) *field_elems = c->g.field;
  return GHB_OK;
}

int64_t ghb_field_elems(const ghb_ctx* c) { return c ? c->g.field : 0; }
int64_t ghb_table_elems(const ghb_ctx* c) { return c ? c->g.table : 0; }
int64_t ghb_grid_elems(const ghb_ctx* c) { return c ? c->g.grid : 0; }
int64_t ghb_device_bytes(const ghb_ctx* c) { return c ? c->bytes : 0; }

ghb_status ghb_matvec(ghb_ctx* c, int kind, int precision, int project, const void* x_dev,
                      void* y_dev, void* stream) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c || !x_dev || !y_dev) { set_error("null argument"); return GHB_ERR_INVALID; }
  if (kind < GHB_PRIMAL || kind > GHB_GANI_DUAL) {
    set_error("kind must be GHB_PRIMAL, GHB_DUAL, GHB_GANI_PRIMAL or GHB_GANI_DUAL");
    return GHB_ERR_INVALID;
  }
  if (x_dev == y_dev) { set_error("x and y must not overlap"); return GHB_ERR_INVALID; }
  if (precision != GHB_FP64 && precision != GHB_FP32) {
    set_error("precision must be GHB_FP64 or GHB_FP32");
    return GHB_ERR_INVALID;
  }
  cudaStream_t saved = c->stream;
  if (stream) c->stream = static_cast<cudaStream_t>(stream);
  const int k = kind & 1;
  auto run = [&]() -> ghb_status {
    if (precision == GHB_FP64)
      return apply_op<double2>(c, k, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev), project != 0);
    return apply_op<float2>(c, k, static_cast<const float2*>(x_dev), static_cast<float2*>(y_dev), project != 0);
  };
  const ghb_status s = kind >= GHB_GANI_PRIMAL ? with_gani(c, run) : run();
  c->stream = saved;
  return s;
  ABI_GUARD_END
}

static ghb_status solve_abi(ghb_ctx* c, int kind, const double* E, void* field_out_dev,
                            ghb_solve_info* info) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c || !E) { set_error("null argument"); return GHB_ERR_INVALID; }
  for (int a = 0; a < c->g.d; ++a)
    if (!std::isfinite(E[a])) { set_error("load must be finite"); return GHB_ERR_INVALID; }
  ghb_solve_info inf{};
  TRY(solve(c, kind, E, c->sol[0], &inf));
  const double2* f0 = c->sol[0];
  double en = 0.0;
  TRY(gram(c, *c->op, kind, 1, &f0, &en));
  inf.energy = en;
  if (field_out_dev) {
    GHB_CUDA_TRY(cudaMemcpyAsync(field_out_dev, c->sol[0], sizeof(double2) * c->g.field,
                                 cudaMemcpyDeviceToDevice, c->stream));
    GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  if (info) *info = inf;
  return static_cast<ghb_status>(inf.status);
  ABI_GUARD_END
}

ghb_status ghb_solve_primal(ghb_ctx* c, const double* E, void* field_out_dev, ghb_solve_info* info) {
  return solve_abi(c, GHB_PRIMAL, E, field_out_dev, info);
}

ghb_status ghb_solve_dual(ghb_ctx* c, const double* J, void* field_out_dev, ghb_solve_info* info) {
  return solve_abi(c, GHB_DUAL, J, field_out_dev, info);
}

ghb_status ghb_gram(ghb_ctx* c, int kind, int m, const void* const* fields_dev, double* out) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c || !fields_dev || !out) { set_error("null argument"); return GHB_ERR_INVALID; }
  if (m < 1 || m > 3) { set_error("m must be 1..3"); return GHB_ERR_INVALID; }
  if (m > c->g.d) { set_error("m must not exceed d"); return GHB_ERR_INVALID; }
  const double2* f[3] = {nullptr, nullptr, nullptr};
  for (int i = 0; i < m; ++i) {
    if (!fields_dev[i]) { set_error("null field"); return GHB_ERR_INVALID; }
    f[i] = static_cast<const double2*>(fields_dev[i]);
  }
  return gram(c, c->ga, kind == GHB_DUAL ? 1 : 0, m, f, out);
  ABI_GUARD_END
}

ghb_status ghb_bounds(ghb_ctx* c, double* upper, double* lower, ghb_solve_info* infos) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c || !upper || !lower) { set_error("null argument"); return GHB_ERR_INVALID; }
  const int d = c->g.d;
  ghb_status worst = GHB_OK;
  double G[2][9];
  // Mixed precision: each solve ends with an FP64 operator application to its
  // iterate, whose output before projection gives the Gram matrix on Z_N
  // (launch_gram_zn) without the double-grid Gram passes.
  const bool reuse = c->opt.precision == GHB_MIXED && c->op == &c->ga;
  for (int kind = 0; kind < 2; ++kind) {
    bool all_ax = reuse;
    for (int i = 0; i < d; ++i) {
      double E[3] = {0, 0, 0};
      E[i] = 1.0;
      ghb_solve_info inf{};
      bool ax_ok = false;
      TRY(solve(c, kind, E, c->sol[i], &inf, nullptr, nullptr, reuse ? c->gT1[i] : nullptr,
                &ax_ok));
      all_ax = all_ax && ax_ok;
      if (inf.status != GHB_OK && worst == GHB_OK) worst = static_cast<ghb_status>(inf.status);
      if (infos) infos[kind * d + i] = inf;
    }
    const double2* f[3] = {c->sol[0], c->sol[1], d == 3 ? c->sol[2] : nullptr};
    if (all_ax) {
      GramZnArgs ga{};
      for (int i = 0; i < d; ++i) {
        ga.v[i] = c->sol[i];
        ga.y[i] = c->gT1[i];
      }
      PROF(c, PK_MISC, false,
           launch_gram_zn(ga, c->tab[kind], c->g, c->partials, kMaxPartials * 6, c->d_gram, c->stream));
      GHB_CUDA_TRY(cudaMemcpyAsync(c->h_gram, c->d_gram, sizeof(double) * d * d, cudaMemcpyDeviceToHost,
                                   c->stream));
      GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
      for (int q = 0; q < d * d; ++q) G[kind][q] = c->h_gram[q];
    } else {
      TRY(gram(c, c->ga, kind, d, f, G[kind]));
    }
    if (infos)
      for (int i = 0; i < d; ++i) infos[kind * d + i].energy = G[kind][i * d + i];
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) upper[i * d + j] = 0.5 * (G[0][i * d + j] + G[0][j * d + i]);
  double Ds[9], L[9];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Ds[i * d + j] = 0.5 * (G[1][i * d + j] + G[1][j * d + i]);
  if (!inverse_small(d, Ds, L)) {
    set_error("dual Gram matrix is not positive definite");
    return GHB_ERR_BREAKDOWN;
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) lower[i * d + j] = 0.5 * (L[i * d + j] + L[j * d + i]);
  if (worst != GHB_OK) set_error("a solve did not reach the tolerance (the bounds are still guaranteed)");
  return worst;
  ABI_GUARD_END
}

ghb_status ghb_solve_ex(ghb_ctx* c, int kind, const double* E, const void* x0_dev, void* field_out_dev,
                        ghb_solve_info* info, double* energies, int cap, int* n_energies) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c || !E) { set_error("null argument"); return GHB_ERR_INVALID; }
  if (kind != GHB_PRIMAL && kind != GHB_DUAL) { set_error("kind must be GHB_PRIMAL or GHB_DUAL"); return GHB_ERR_INVALID; }
  if (energies && cap < 1) { set_error("cap must be >= 1 when energies is given"); return GHB_ERR_INVALID; }
  for (int a = 0; a < c->g.d; ++a)
    if (!std::isfinite(E[a])) { set_error("load must be finite"); return GHB_ERR_INVALID; }
  std::vector<double> hist;
  ghb_solve_info inf{};
  TRY(solve(c, kind, E, c->sol[0], &inf, static_cast<const double2*>(x0_dev), energies ? &hist : nullptr));
  const double2* f0 = c->sol[0];
  double en = 0.0;
  TRY(gram(c, c->ga, kind, 1, &f0, &en));
  inf.energy = en;
  if (field_out_dev) {
    GHB_CUDA_TRY(cudaMemcpyAsync(field_out_dev, c->sol[0], sizeof(double2) * c->g.field,
                                 cudaMemcpyDeviceToDevice, c->stream));
    GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  if (energies) {
    const int n = static_cast<int>(std::min<size_t>(hist.size(), static_cast<size_t>(cap)));
    for (int i = 0; i < n; ++i) energies[i] = hist[i];
    if (n_energies) *n_energies = n;
  } else if (n_energies) {
    *n_energies = 0;
  }
  if (info) *info = inf;
  if (inf.status != GHB_OK) set_error("the solve did not reach the tolerance (the bound is still guaranteed)");
  return static_cast<ghb_status>(inf.status);
  ABI_GUARD_END
}

ghb_status ghb_prolong(int d, const int* Nc, const void* xc_dev, const int* Nf, void* xf_dev, void* stream) {
  clear_error();
  if ((d != 2 && d != 3) || !Nc || !Nf || !xc_dev || !xf_dev) {
    set_error("ghb_prolong: d must be 2 or 3 and no pointer may be NULL");
    return GHB_ERR_INVALID;
  }
  int nc[3] = {1, 1, 1}, nf[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) {
    if (Nc[a] < 1 || Nc[a] % 2 == 0 || Nf[a] < Nc[a] || Nf[a] % 2 == 0) {
      set_error("ghb_prolong: orders must be odd with N_fine >= N_coarse in every direction");
      return GHB_ERR_INVALID;
    }
    nc[a] = Nc[a];
    nf[a] = Nf[a];
  }
  const int hc = (nc[d - 1] + 1) / 2, hf = (nf[d - 1] + 1) / 2;
  int64_t Pc = hc, Pf = hf;
  for (int a = 0; a < d - 1; ++a) {
    Pc *= nc[a];
    Pf *= nf[a];
  }
  const FieldGeom fc = make_field_geom(d, nc[0], nc[1], nc[2], hc, Pc);
  const FieldGeom ff = make_field_geom(d, nf[0], nf[1], nf[2], hf, Pf);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TRY(launch_prolong(static_cast<double2*>(xf_dev), ff, static_cast<const double2*>(xc_dev), fc, s));
  GHB_CUDA_TRY(cudaStreamSynchronize(s));
  return GHB_OK;
}

ghb_status ghb_bounds_gani(ghb_ctx* c, double* upper, double* lower, double* a_gani, double* b_gani_inv,
                           ghb_solve_info* infos) {
  ABI_GUARD_BEGIN
  clear_error();
  if (!c || !upper || !lower) { set_error("null argument"); return GHB_ERR_INVALID; }
  const int d = c->g.d;
  ghb_status worst = GHB_OK;
  double Gx[2][9], Gn[2][9];
  for (int kind = 0; kind < 2; ++kind) {
    TRY(with_gani(c, [&]() -> ghb_status {
      for (int i = 0; i < d; ++i) {
        double E[3] = {0, 0, 0};
        E[i] = 1.0;
        ghb_solve_info inf{};
        TRY(solve(c, kind, E, c->sol[i], &inf));
        if (inf.status != GHB_OK && worst == GHB_OK) worst = static_cast<ghb_status>(inf.status);
        if (infos) infos[kind * d + i] = inf;
      }
      return GHB_OK;
    }));
    const double2* f[3] = {c->sol[0], c->sol[1], d == 3 ? c->sol[2] : nullptr};
    TRY(gram(c, c->ga, kind, d, f, Gx[kind]));     // exact energies (eq. GaNi_apost)
    TRY(gram(c, c->gani, kind, d, f, Gn[kind]));   // trapezoidal energies (Def. GaNi)
    if (infos)
      for (int i = 0; i < d; ++i) infos[kind * d + i].energy = Gx[kind][i * d + i];
  }
  auto sym = [&](const double* X, double* Y) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) Y[i * d + j] = 0.5 * (X[i * d + j] + X[j * d + i]);
  };
  auto inv_sym = [&](const double* X, double* Y) -> bool {
    double S[9] = {}, L[9] = {};
    sym(X, S);
    if (!inverse_small(d, S, L)) return false;
    sym(L, Y);
    return true;
  };
  sym(Gx[0], upper);
  if (!inv_sym(Gx[1], lower)) {
    set_error("dual Gram matrix is not positive definite");
    return GHB_ERR_BREAKDOWN;
  }
  if (a_gani) sym(Gn[0], a_gani);
  if (b_gani_inv && !inv_sym(Gn[1], b_gani_inv)) {
    set_error("dual GaNi matrix is not positive definite");
    return GHB_ERR_BREAKDOWN;
  }
  if (worst != GHB_OK) set_error("a solve did not reach the tolerance (the bounds are still guaranteed)");
  return worst;
  ABI_GUARD_END
}

ghb_status ghb_copy_table(ghb_ctx* c, int kind, void* out_dev) {
  clear_error();
  if (!c || !out_dev) { set_error("null argument"); return GHB_ERR_INVALID; }
  GHB_CUDA_TRY(cudaMemcpyAsync(out_dev, c->tab[kind == GHB_DUAL ? 1 : 0], sizeof(double2) * c->g.table,
                               cudaMemcpyDeviceToDevice, c->stream));
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return GHB_OK;
}

ghb_status ghb_copy_grid_values(ghb_ctx* c, int kind, void* out_dev) {
  clear_error();
  if (!c || !out_dev) { set_error("null argument"); return GHB_ERR_INVALID; }
  GHB_CUDA_TRY(cudaMemcpyAsync(out_dev, c->grid64[kind == GHB_DUAL ? 1 : 0], sizeof(double) * c->g.grid,
                               cudaMemcpyDeviceToDevice, c->stream));
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return GHB_OK;
}

ghb_status ghb_profile(ghb_ctx* c, int enable) {
  clear_error();
  if (!c) { set_error("ctx is NULL"); return GHB_ERR_INVALID; }
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->prof = enable != 0;
  c->nrec = 0;
  return GHB_OK;
}

ghb_status ghb_profile_read(ghb_ctx* c, int cls, int64_t* launches, double* total_ms,
                            double* bytes_per_launch, double* flops_per_launch) {
  clear_error();
  if (!c) { set_error("ctx is NULL"); return GHB_ERR_INVALID; }
  if (cls < 0 || cls >= 2 * PK_COUNT) { set_error("profile class out of range"); return GHB_ERR_INVALID; }
  GHB_CUDA_TRY(cudaStreamSynchronize(c->stream));
  int64_t n = 0;
  double ms = 0.0;
  for (int i = 0; i < c->nrec; ++i) {
    if (c->rec_cls[i] != cls) continue;
    float t = 0.f;
    GHB_CUDA_TRY(cudaEventElapsedTime(&t, c->ev[2 * i], c->ev[2 * i + 1]));
    ms += t;
    ++n;
  }
  double b = 0, f = 0;
  algo_model(c, cls / 2, (cls % 2) == 1, &b, &f);
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (bytes_per_launch) *bytes_per_launch = b;
  if (flops_per_launch) *flops_per_launch = f;
  return GHB_OK;
}

void ghb_destroy(ghb_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

}  // extern "C"
