// Batched and continuously served Ga bound computations (C ABI ghb_batch_*).
//
// Many requests -- each one microstructure at its own order N, asking for the
// d x d upper and lower bounds (Def. Ga, Prop. struct_bounds) -- are solved
// together.  Every request becomes an instance with 2d solves (d primal, d
// dual loads).  Each CG iteration is one launch per kernel over all active
// solves (work items of uneven size, see ColItem / RowItem / CgItem), in the
// mixed scheme of the single-instance path: FP32 inner CG, FP64 residual
// correction, exact FP64 projection, FP64 Gram energies.
//
// The engine is a loop of cycles (ghb_batch_step):
//   admit     pending requests while the device-memory budget allows
//             (coefficient set-up, right-hand sides, inner CG start),
//   iterate   K batched FP32 CG iterations over every solve in its inner phase
//             (solves whose inner CG has ended return at once from each kernel);
//             one iteration's launches are captured as a CUDA graph and replayed,
//   correct   batched FP64 correction of the solves whose inner CG ended:
//             x64 = G(x64 + dx), r64 = b - G A x64; stop or restart the inner CG,
//   retire    batched Gram energies of the instances whose solves all ended;
//             their results become available and their memory returns to the pool.
// Requests submitted while others run are admitted at the next cycle, so work
// of requests of different ages overlaps on the device (continuous batching).
//
// Large requests (at least kLargeGrid double-grid points) do not enter the
// batched cycles: every batched launch advances all active solves together,
// so one large solve would set the pace of every iteration for all the small
// ones.  A worker thread solves them one at a time with a private context
// (ghb_create / ghb_bounds on the context's own stream: size-specialised,
// autotuned kernels) while the cycles run, two at a time; their results join
// the same queue.
// The context's device memory counts against the batch's budget while it
// exists.  Context set-up and teardown (which allocate and copy synchronously)
// never overlap the capture of a cycle's CUDA graph.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ghb_internal.cuh"

namespace ghb {
const char* last_error_cstr();
void clear_error();
}  // namespace ghb

using namespace ghb;

namespace {

#define TRYB(expr)                     \
  do {                                 \
    ghb_status s__ = (expr);           \
    if (s__ != GHB_OK) return s__;     \
  } while (0)

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum SlotState { S_INNER = 0, S_DONE = 1 };

struct Inst;

struct Slot {
  Inst* inst = nullptr;
  int kind = 0;
  int load = 0;
  int sidx = -1;            // index of this solve's CgState
  int state = S_INNER;
  float2 *x32, *r32, *p32, *q32, *w32, *b32, *T1_32, *T2_32;
  double2 *x64, *xacc, *r64, *b64, *y64, *w64, *T1_64, *T2_64, *sol;
  double* partials;
  double bb = 0.0;
  int inner_iters = 0, outer = 0, mv32 = 0, mv64 = 0;
  double relres = 0.0;
  int status = GHB_OK;
};

struct Inst {
  int64_t id = 0;
  Geometry g{};
  FftPlan hpl[3];
  const FftPlan* dpl[3] = {nullptr, nullptr, nullptr};
  char* block = nullptr;
  int64_t bytes = 0;
  double2* tab[2];
  double* grid64[2];
  float* grid32[2];
  double2* tabT1;
  double2* tabT2;
  Incl* incs;
  double* gram_partials[2];
  unsigned int* gram_ticket;
  double* gram_d;           // 2 x 9
  int nslots = 0;
  Slot slots[6];
  double t_submit = 0, t_admit = 0;
};

struct Request {
  int64_t id;
  int d;
  int N[3];
  double a0;
  std::vector<ghb_phase> phases;
  double t_submit;
};

struct PlanEntry {
  PlanHolder h;
  FftPlan* d_plan = nullptr;
};

FieldGeom fgeom_of(const Geometry& g) { return make_field_geom(g.d, g.N[0], g.N[1], g.N[2], g.h, g.P); }

// Work-item arrays of the launches of one phase: appended to a pinned host
// buffer, copied to the device with one transfer (flush) before the launches
// that read them, and reset only after a stream synchronisation (when no queued
// kernel can still read them).
struct Arena {
  char* h = nullptr;
  char* d = nullptr;
  size_t cap = 0, used = 0, flushed = 0;
  ghb_status init(size_t bytes) {
    GHB_CUDA_TRY(cudaMallocHost(&h, bytes));
    GHB_CUDA_TRY(cudaMalloc(&d, bytes));
    cap = bytes;
    return GHB_OK;
  }
  template <typename Item>
  ghb_status push(const std::vector<Item>& v, const Item** dev) {
    const size_t bytes = sizeof(Item) * v.size();
    const size_t off = (used + 255) & ~static_cast<size_t>(255);
    if (off + bytes > cap) {
      set_error("batch work-item arena exhausted");
      return GHB_ERR_OOM;
    }
    std::memcpy(h + off, v.data(), bytes);
    used = off + bytes;
    *dev = reinterpret_cast<const Item*>(d + off);
    return GHB_OK;
  }
  ghb_status flush(cudaStream_t s) {
    if (used > flushed) {
      GHB_CUDA_TRY(cudaMemcpyAsync(d + flushed, h + flushed, used - flushed, cudaMemcpyHostToDevice, s));
      flushed = used;
    }
    return GHB_OK;
  }
  void reset() { used = flushed = 0; }
  void release() {
    if (h) cudaFreeHost(h);
    if (d) cudaFree(d);
    h = d = nullptr;
  }
};

// A prepared batched launch.
struct Launch {
  int kind;             // 0 col, 1 row, 2 cg
  bool f32;
  int sign, mode, op, tile;   // tile: TW (col) or NL (row)
  int threads;                // threads per CTA (0 = the kernel's full block)
  const void* items;
  int n;
  int64_t blocks;
  size_t smem;
};

}  // namespace

// Double-grid points from which a request is solved by the large-request
// worker instead of the batched cycles (2^22: d = 3 from M = 162, d = 2 from
// M = 2048).
constexpr int64_t kLargeGrid = int64_t(1) << 22;

// Large requests solved at the same time (each by its own worker thread and
// context): two, so that one solve's launch gaps and barrier waits are filled
// by the other's kernels.
constexpr int kLaneWorkers = 2;

struct LargeLane {
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> queue;
  std::deque<ghb_result> done;
  bool stop = false;
  int running = 0;
  int device = 0;
};

struct ghb_batch {
  ghb_options opt{};
  cudaStream_t stream = nullptr;
  int64_t budget = 0;
  std::atomic<int64_t> in_use{0};
  LargeLane lane;
  std::mutex capture_mu;   // held while a cycle's graph is captured
  int max_active = 0;
  int64_t next_id = 1;
  std::map<int, PlanEntry> plans;
  std::deque<Request> pending;
  std::vector<Inst*> active;
  std::deque<ghb_result> results;
  int64_t finished = 0;
  // solve states
  int cap_states = 0;
  CgState* d_states = nullptr;
  CgState* h_states = nullptr;
  std::vector<int> free_states;
  Arena arena;
  int64_t launches = 0;
  // one inner CG iteration's launches of the current cycle, captured once and
  // replayed; destroyed after the next stream synchronisation
  cudaGraphExec_t graph = nullptr;
};

namespace {

ghb_status get_plan(ghb_batch* b, int M, const FftPlan** dpl, FftPlan* hpl) {
  auto it = b->plans.find(M);
  if (it == b->plans.end()) {
    PlanEntry e;
    TRYB(make_plan(M, e.h));
    GHB_CUDA_TRY(cudaMalloc(&e.d_plan, sizeof(FftPlan)));
    GHB_CUDA_TRY(cudaMemcpy(e.d_plan, &e.h.plan, sizeof(FftPlan), cudaMemcpyHostToDevice));
    it = b->plans.emplace(M, e).first;
  }
  *dpl = it->second.d_plan;
  *hpl = it->second.h.plan;
  return GHB_OK;
}

int64_t align256(int64_t n) { return (n + 255) & ~static_cast<int64_t>(255); }

// Layout of one instance's device block; when `base` is null only the size is computed.
int64_t layout_instance(Inst* in, char* base, int nphases) {
  const Geometry& g = in->g;
  const int d = g.d;
  int64_t off = 0;
  auto take = [&](int64_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  for (int k = 0; k < 2; ++k) in->tab[k] = reinterpret_cast<double2*>(take(16 * g.table));
  for (int k = 0; k < 2; ++k) in->grid64[k] = reinterpret_cast<double*>(take(8 * g.grid));
  for (int k = 0; k < 2; ++k) in->grid32[k] = reinterpret_cast<float*>(take(4 * g.grid));
  int64_t t1tab, t2tab = 0;
  if (d == 2) {
    t1tab = static_cast<int64_t>(g.M[0]) * g.N[1];
  } else {
    t1tab = static_cast<int64_t>(g.M[0]) * (2 * g.N[1] - 1) * g.N[2];
    t2tab = static_cast<int64_t>(g.M[0]) * g.M[1] * g.N[2];
  }
  in->tabT1 = reinterpret_cast<double2*>(take(16 * t1tab));
  in->tabT2 = reinterpret_cast<double2*>(take(16 * std::max<int64_t>(t2tab, 1)));
  in->incs = reinterpret_cast<Incl*>(take(sizeof(Incl) * 2 * std::max(nphases, 1)));
  for (int k = 0; k < 2; ++k) in->gram_partials[k] = reinterpret_cast<double*>(take(8 * 1024 * 6));
  in->gram_ticket = reinterpret_cast<unsigned int*>(take(64));
  in->gram_d = reinterpret_cast<double*>(take(8 * 18));
  const int64_t F = g.field;
  const int64_t nb = cg_blocks(fgeom_of(g));
  for (int s = 0; s < 2 * d; ++s) {
    Slot& sl = in->slots[s];
    sl.x32 = reinterpret_cast<float2*>(take(8 * F));
    sl.r32 = reinterpret_cast<float2*>(take(8 * F));
    sl.p32 = reinterpret_cast<float2*>(take(8 * F));
    sl.q32 = reinterpret_cast<float2*>(take(8 * F));
    sl.w32 = reinterpret_cast<float2*>(take(8 * F));
    sl.b32 = reinterpret_cast<float2*>(take(8 * F));
    sl.T1_32 = reinterpret_cast<float2*>(take(8 * g.T1));
    sl.T2_32 = reinterpret_cast<float2*>(take(8 * std::max<int64_t>(g.T2, 1)));
    sl.x64 = reinterpret_cast<double2*>(take(16 * F));
    sl.xacc = reinterpret_cast<double2*>(take(16 * F));
    sl.r64 = reinterpret_cast<double2*>(take(16 * F));
    sl.b64 = reinterpret_cast<double2*>(take(16 * F));
    sl.y64 = reinterpret_cast<double2*>(take(16 * F));
    sl.w64 = reinterpret_cast<double2*>(take(16 * F));
    sl.T1_64 = reinterpret_cast<double2*>(take(16 * g.T1));
    sl.T2_64 = reinterpret_cast<double2*>(take(16 * std::max<int64_t>(g.T2, 1)));
    sl.sol = reinterpret_cast<double2*>(take(16 * F));
    sl.partials = reinterpret_cast<double*>(take(8 * nb));
  }
  return off;
}

ghb_status make_geometry(int d, const int* N, const ghb_options& o, Geometry* out) {
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
    if (M < 2 * N[a] - 1 || M > (d == 2 ? 6400 : 2560) || !factorizable(M)) {
      set_error("unsupported double grid M=" + std::to_string(M));
      return GHB_ERR_INVALID;
    }
    g.M[a] = M;
  }
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
  *out = g;
  return GHB_OK;
}

// Coefficient tables and double-grid values of one instance (eq.
// inclcomp_formula, eq. MBA_GA), with the same one-operand launches as a context.
ghb_status setup_coeffs(ghb_batch* b, Inst* in, const Request& rq) {
  const Geometry& g = in->g;
  const int n = static_cast<int>(rq.phases.size());
  std::vector<Incl> h(2 * std::max(n, 1));
  for (int kind = 0; kind < 2; ++kind) {
    const double a0v = kind == 0 ? rq.a0 : 1.0 / rq.a0;
    for (int i = 0; i < n; ++i) {
      Incl& ic = h[kind * n + i];
      ic.shape = rq.phases[i].shape;
      ic.pad = 0;
      for (int a = 0; a < 3; ++a) {
        ic.c[a] = a < g.d ? rq.phases[i].center[a] : 0.0;
        ic.s[a] = rq.phases[i].size[a];
      }
      const double v = kind == 0 ? rq.phases[i].value : 1.0 / rq.phases[i].value;
      ic.dv = v - a0v;
      ic.v = v;
    }
  }
  // stream-ordered: the block was allocated on this stream (pageable source, staged before return)
  if (n > 0)
    GHB_CUDA_TRY(cudaMemcpyAsync(in->incs, h.data(), sizeof(Incl) * 2 * n, cudaMemcpyHostToDevice, b->stream));
  // both tables in one pass (shared shape factors and phases)
  TRYB(launch_coeff_tables(in->tab[0], in->tab[1], g, in->incs, in->incs + n, n, rq.a0, 1.0 / rq.a0, b->stream));
  for (int kind = 0; kind < 2; ++kind) {
    const int Nd = g.N[g.d - 1];
    if (g.d == 2) {
      ColArgs a{};
      a.in = in->tab[kind];
      a.out = in->tabT1;
      a.outer = 1;
      a.inner = Nd;
      a.Lin = 2 * g.N[0] - 1;
      a.Lout = g.M[0];
      TRYB(launch_col<double>(+1, COL_PLAIN, a, in->hpl[0], b->stream));
      RowArgs r{};
      r.t[0] = in->tabT1;
      r.nfields = 1;
      r.ncomp = 1;
      r.rows = g.M[0];
      r.H = Nd;
      r.out_real = in->grid64[kind];
      TRYB(launch_row<double>(ROW_TOREAL, r, in->hpl[1], b->stream));
    } else {
      ColArgs a{};
      a.in = in->tab[kind];
      a.out = in->tabT1;
      a.outer = 1;
      a.inner = static_cast<int64_t>(2 * g.N[1] - 1) * Nd;
      a.Lin = 2 * g.N[0] - 1;
      a.Lout = g.M[0];
      TRYB(launch_col<double>(+1, COL_PLAIN, a, in->hpl[0], b->stream));
      ColArgs c{};
      c.in = in->tabT1;
      c.out = in->tabT2;
      c.outer = g.M[0];
      c.inner = Nd;
      c.Lin = 2 * g.N[1] - 1;
      c.Lout = g.M[1];
      TRYB(launch_col<double>(+1, COL_PLAIN, c, in->hpl[1], b->stream));
      RowArgs r{};
      r.t[0] = in->tabT2;
      r.nfields = 1;
      r.ncomp = 1;
      r.rows = static_cast<int64_t>(g.M[0]) * g.M[1];
      r.H = Nd;
      r.out_real = in->grid64[kind];
      TRYB(launch_row<double>(ROW_TOREAL, r, in->hpl[2], b->stream));
    }
    TRYB(launch_to_f32_real(in->grid32[kind], in->grid64[kind], g.grid, b->stream));
  }
  return GHB_OK;
}

CgItem cg_item(const Slot& s) {
  CgItem it{};
  it.fg = fgeom_of(s.inst->g);
  it.st = nullptr;
  it.nblocks = cg_blocks(it.fg);
  it.kind = s.kind;
  return it;
}

// Prepare one batched CG op over items (block ranges assigned here).
template <typename T>
ghb_status prep_cg(ghb_batch* b, int op, std::vector<CgItem>& items, std::vector<Launch>& out) {
  if (items.empty()) return GHB_OK;
  int64_t blocks = 0;
  for (auto& it : items) {
    it.block_begin = blocks;
    blocks += it.nblocks;
  }
  Launch L{};
  L.kind = 2;
  L.f32 = sizeof(T) == 4;
  L.op = op;
  L.n = static_cast<int>(items.size());
  L.blocks = blocks;
  const CgItem* dp = nullptr;
  TRYB(b->arena.push(items, &dp));
  L.items = dp;
  out.push_back(L);
  return GHB_OK;
}

// Threads per CTA of a batched transform pass over `lines` interleaved lines
// of length at most Mmax: about one thread per butterfly of a pass (a pass
// combines up to 32 entries in FP32 and 18 in FP64, so a line has at least
// Mmax / 32 or Mmax / 18 of them), in whole warps, at least 64.  Short
// transforms then run several CTAs per SM instead of one CTA whose threads
// mostly wait.
template <typename T>
int batch_threads(int Mmax, int lines, int full) {
  const int cap = sizeof(T) == 4 ? 32 : 18;
  const int units = (Mmax + cap - 1) / cap;
  int t = ((units * lines + 31) / 32) * 32;
  if (t < 64) t = 64;
  return t < full ? t : full;
}

template <typename T>
ghb_status prep_col(ghb_batch* b, int sign, int mode, std::vector<ColItem>& items, const std::vector<int>& Ms,
                    std::vector<Launch>& out) {
  if (items.empty()) return GHB_OK;
  using C = typename CT<T>::type;
  int Mmax = 1;
  for (int M : Ms) Mmax = std::max(Mmax, M);
  // Launch shapes of the batched passes follow the size rules: the
  // autotuner's tile widths are timed on one operand and measured slower for
  // launches over many items of mixed lengths.  The items' radix groupings
  // (their plans) are the tuned ones.
  const int TW = col_tile_width(Mmax, sizeof(C));
  int64_t blocks = 0;
  for (auto& it : items) {
    it.block_begin = blocks;
    blocks += ((it.a.inner + TW - 1) / TW) * it.a.outer;
  }
  Launch L{};
  L.kind = 0;
  L.f32 = sizeof(T) == 4;
  L.sign = sign;
  L.mode = mode;
  L.tile = TW;
  L.threads = batch_threads<T>(Mmax, TW, sizeof(T) == 4 ? 512 : 256);
  L.n = static_cast<int>(items.size());
  L.blocks = blocks;
  L.smem = col_smem_bytes(Mmax, TW, sizeof(C));
  const ColItem* dp = nullptr;
  TRYB(b->arena.push(items, &dp));
  L.items = dp;
  out.push_back(L);
  return GHB_OK;
}

template <typename T>
ghb_status prep_row(ghb_batch* b, int mode, std::vector<RowItem>& items, const std::vector<int>& Ms, int nfields,
                    int ncomp, std::vector<Launch>& out) {
  if (items.empty()) return GHB_OK;
  using C = typename CT<T>::type;
  int Mmax = 1;
  for (int M : Ms) Mmax = std::max(Mmax, M);
  int rpc = 1, NL = 1;
  row_lines(mode, nfields, ncomp, Mmax, 0, &rpc, &NL);
  int64_t blocks = 0;
  for (auto& it : items) {
    it.rows_per_cta = rpc;
    const int64_t groups = (it.a.rows + rpc - 1) / rpc;
    it.nblocks = (mode == ROW_ENERGY) ? std::min<int64_t>(groups, 1024) : groups;
    it.block_begin = blocks;
    blocks += it.nblocks;
  }
  Launch L{};
  L.kind = 1;
  L.f32 = sizeof(T) == 4;
  L.mode = mode;
  L.tile = NL;
  L.threads = mode == ROW_MATVEC ? batch_threads<T>(Mmax, NL, 256) : 0;
  L.n = static_cast<int>(items.size());
  L.blocks = blocks;
  L.smem = padded_elems<C>(static_cast<size_t>(Mmax) * NL) * sizeof(C);
  const RowItem* dp = nullptr;
  TRYB(b->arena.push(items, &dp));
  L.items = dp;
  out.push_back(L);
  return GHB_OK;
}

ghb_status run_launch(ghb_batch* b, const Launch& L) {
  ++b->launches;
  if (L.kind == 0) {
    const ColItem* it = static_cast<const ColItem*>(L.items);
    return L.f32 ? launch_col_batch<float>(L.sign, L.mode, L.tile, it, L.n, L.blocks, L.smem, L.threads, b->stream)
                 : launch_col_batch<double>(L.sign, L.mode, L.tile, it, L.n, L.blocks, L.smem, L.threads, b->stream);
  }
  if (L.kind == 1) {
    const RowItem* it = static_cast<const RowItem*>(L.items);
    return L.f32 ? launch_row_batch<float>(L.mode, L.tile, it, L.n, L.blocks, L.smem, L.threads, b->stream)
                 : launch_row_batch<double>(L.mode, L.tile, it, L.n, L.blocks, L.smem, L.threads, b->stream);
  }
  const CgItem* it = static_cast<const CgItem*>(L.items);
  return L.f32 ? launch_cg_batch<float>(L.op, it, L.n, L.blocks, b->stream)
               : launch_cg_batch<double>(L.op, it, L.n, L.blocks, b->stream);
}

ghb_status run_all(ghb_batch* b, const std::vector<Launch>& v) {
  TRYB(b->arena.flush(b->stream));
  for (const Launch& L : v) TRYB(run_launch(b, L));
  return GHB_OK;
}

// One batched operator application y = A^full x (not projected) for the given
// solves, FP32 (inner CG, with the direction update p = r + beta p fused in
// the first pass) or FP64 (correction).  Outputs: w32 / w64 of every solve.
template <typename T>
ghb_status prep_operator(ghb_batch* b, const std::vector<Slot*>& ss, bool cg, std::vector<Launch>& out) {
  using C = typename CT<T>::type;
  constexpr bool f32 = sizeof(T) == 4;
  for (int d = 2; d <= 3; ++d) {
    std::vector<ColItem> c1, c2, f2, f1;
    std::vector<RowItem> rw;
    std::vector<int> M0, M1, Md;
    for (Slot* s : ss) {
      if (s->inst->g.d != d) continue;
      const Geometry& g = s->inst->g;
      C* T1 = f32 ? reinterpret_cast<C*>(s->T1_32) : reinterpret_cast<C*>(s->T1_64);
      C* T2 = f32 ? reinterpret_cast<C*>(s->T2_32) : reinterpret_cast<C*>(s->T2_64);
      const CgState* st = (f32 && cg) ? &b->d_states[s->sidx] : nullptr;
      ColItem a{};
      a.a.in = f32 ? static_cast<const void*>(s->r32) : static_cast<const void*>(s->x64);
      a.a.out = T1;
      a.a.pold = f32 ? s->p32 : nullptr;
      a.a.pnew = f32 ? s->p32 : nullptr;
      a.a.st = st;
      a.a.outer = d;
      a.a.inner = g.P / g.N[0];
      a.a.Lin = g.N[0];
      a.a.Lout = g.M[0];
      a.pl = s->inst->dpl[0];
      c1.push_back(a);
      M0.push_back(g.M[0]);
      C* last = T1;
      if (d == 3) {
        ColItem c{};
        c.a.in = T1;
        c.a.out = T2;
        c.a.st = st;
        c.a.outer = static_cast<int64_t>(d) * g.M[0];
        c.a.inner = g.h;
        c.a.Lin = g.N[1];
        c.a.Lout = g.M[1];
        c.pl = s->inst->dpl[1];
        c2.push_back(c);
        M1.push_back(g.M[1]);
        ColItem f{};
        f.a.in = T2;
        f.a.out = T1;
        f.a.st = st;
        f.a.outer = static_cast<int64_t>(d) * g.M[0];
        f.a.inner = g.h;
        f.a.Lin = g.M[1];
        f.a.Lout = g.N[1];
        f.pl = s->inst->dpl[1];
        f2.push_back(f);
        last = T2;
      }
      RowItem r{};
      r.a.t[0] = last;
      r.a.nfields = 1;
      r.a.ncomp = d;
      r.a.rows = g.rows;
      r.a.H = g.h;
      r.a.comp_stride = g.rows * g.h;
      r.a.a = f32 ? static_cast<const void*>(s->inst->grid32[s->kind])
                  : static_cast<const void*>(s->inst->grid64[s->kind]);
      r.a.st = st;
      r.pl = s->inst->dpl[d - 1];
      rw.push_back(r);
      Md.push_back(g.M[d - 1]);
      ColItem o{};
      o.a.in = T1;
      o.a.out = f32 ? static_cast<void*>(s->w32) : static_cast<void*>(s->w64);
      o.a.st = st;
      o.a.outer = d;
      o.a.inner = g.P / g.N[0];
      o.a.Lin = g.M[0];
      o.a.Lout = g.N[0];
      o.pl = s->inst->dpl[0];
      f1.push_back(o);
    }
    TRYB(prep_col<T>(b, +1, (f32 && cg) ? COL_PUPDATE : COL_PLAIN, c1, M0, out));
    TRYB(prep_col<T>(b, +1, COL_PLAIN, c2, M1, out));
    TRYB(prep_row<T>(b, ROW_MATVEC, rw, Md, 1, d, out));
    TRYB(prep_col<T>(b, -1, COL_PLAIN, f2, M1, out));
    TRYB(prep_col<T>(b, -1, COL_PLAIN, f1, M0, out));
  }
  return GHB_OK;
}

ghb_status read_states(ghb_batch* b) {
  int hi = 0;
  for (Inst* in : b->active)
    for (int s = 0; s < in->nslots; ++s) hi = std::max(hi, in->slots[s].sidx + 1);
  if (hi == 0) return GHB_OK;
  GHB_CUDA_TRY(cudaMemcpyAsync(b->h_states, b->d_states, sizeof(CgState) * hi, cudaMemcpyDeviceToHost,
                               b->stream));
  GHB_CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->arena.reset();
  if (b->graph) {   // its replays have completed
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return GHB_OK;
}

// Start (or restart) the FP32 inner CG of the given solves on b32 = f32(r64).
ghb_status start_inner(ghb_batch* b, const std::vector<Slot*>& ss) {
  std::vector<CgItem> conv, init;
  for (Slot* s : ss) {
    CgItem c = cg_item(*s);
    c.q = s->b32;
    c.w = s->r64;
    conv.push_back(c);
    CgItem i = cg_item(*s);
    i.x = s->x32;
    i.r = s->r32;
    i.p = s->p32;
    i.b = s->b32;
    i.st = &b->d_states[s->sidx];
    i.partials = s->partials;
    i.tol = inner_target(b->opt.inner_tol, b->opt.tol, b->h_states[s->sidx].rr, s->bb);
    i.maxiter = std::max(1, b->opt.max_iter - s->inner_iters);
    init.push_back(i);
  }
  std::vector<Launch> L;
  TRYB(prep_cg<double>(b, CG_TO_F32, conv, L));
  TRYB(prep_cg<float>(b, CG_INIT, init, L));
  return run_all(b, L);
}

ghb_status admit(ghb_batch* b) {
  std::vector<Slot*> fresh;
  while (!b->pending.empty() && static_cast<int>(b->active.size()) < b->max_active) {
    const Request& rq = b->pending.front();
    std::unique_ptr<Inst> in(new Inst());
    in->id = rq.id;
    in->t_submit = rq.t_submit;
    TRYB(make_geometry(rq.d, rq.N, b->opt, &in->g));
    const int64_t bytes = layout_instance(in.get(), nullptr, static_cast<int>(rq.phases.size()));
    if (b->in_use + bytes > b->budget) {
      if (b->active.empty()) {
        set_error("request " + std::to_string(rq.id) + " needs " + std::to_string(bytes) +
                  " bytes, more than the batch's device-memory budget");
        b->pending.pop_front();
        ghb_result r{};
        r.id = rq.id;
        r.d = rq.d;
        r.status = GHB_ERR_OOM;
        b->results.push_back(r);
        ++b->finished;
        continue;
      }
      break;   // wait until running requests retire
    }
    // free CgState indices
    if (static_cast<int>(b->free_states.size()) < 2 * rq.d) break;
    for (int a = 0; a < rq.d; ++a) TRYB(get_plan(b, in->g.M[a], &in->dpl[a], &in->hpl[a]));
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&in->block), bytes, b->stream);
    if (e != cudaSuccess) {
      if (b->active.empty()) {
        set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        return GHB_ERR_OOM;
      }
      cudaGetLastError();
      break;
    }
    in->bytes = bytes;
    b->in_use += bytes;
    layout_instance(in.get(), in->block, static_cast<int>(rq.phases.size()));
    in->t_admit = now_s();
    TRYB(setup_coeffs(b, in.get(), rq));
    in->nslots = 2 * rq.d;
    for (int s = 0; s < in->nslots; ++s) {
      Slot& sl = in->slots[s];
      sl.inst = in.get();
      sl.kind = s < rq.d ? GHB_PRIMAL : GHB_DUAL;
      sl.load = s % rq.d;
      sl.sidx = b->free_states.back();
      b->free_states.pop_back();
      sl.state = S_INNER;
      double E[3] = {0, 0, 0};
      E[sl.load] = 1.0;
      TRYB(launch_rhs<double>(sl.b64, in->tab[sl.kind], in->g, E, sl.kind, b->stream));
      GHB_CUDA_TRY(cudaMemsetAsync(sl.x64, 0, 16 * in->g.field, b->stream));
      GHB_CUDA_TRY(cudaMemsetAsync(sl.y64, 0, 16 * in->g.field, b->stream));
      fresh.push_back(&sl);
    }
    b->active.push_back(in.release());
    b->pending.pop_front();
  }
  if (fresh.empty()) return GHB_OK;
  // r64 = b64 - 0 and bb = <b, b>
  std::vector<CgItem> res;
  for (Slot* s : fresh) {
    CgItem c = cg_item(*s);
    c.r = s->r64;
    c.b = s->b64;
    c.w = s->y64;
    c.st = &b->d_states[s->sidx];
    c.partials = s->partials;
    res.push_back(c);
  }
  {
    std::vector<Launch> L;
    TRYB(prep_cg<double>(b, CG_RESIDUAL, res, L));
    TRYB(run_all(b, L));
  }
  TRYB(read_states(b));
  std::vector<Slot*> go;
  for (Slot* s : fresh) {
    s->bb = b->h_states[s->sidx].rr;
    if (s->bb == 0.0) {   // nothing to solve: e = 0 is the minimiser
      s->state = S_DONE;
      double E[3] = {0, 0, 0};
      E[s->load] = 1.0;
      const FieldGeom fg = fgeom_of(s->inst->g);
      TRYB(launch_add_constant(s->sol, s->x64, fg, E, b->stream));
    } else {
      go.push_back(s);
    }
  }
  return start_inner(b, go);
}

ghb_status iterate(ghb_batch* b, int K) {
  std::vector<Slot*> inner;
  for (Inst* in : b->active)
    for (int s = 0; s < in->nslots; ++s)
      if (in->slots[s].state == S_INNER) inner.push_back(&in->slots[s]);
  if (inner.empty()) return GHB_OK;
  std::vector<CgItem> pd, up;
  for (Slot* s : inner) {
    CgItem a = cg_item(*s);
    a.q = s->q32;
    a.w = s->w32;
    a.p = s->p32;
    a.st = &b->d_states[s->sidx];
    a.partials = s->partials;
    pd.push_back(a);
    CgItem u = cg_item(*s);
    u.x = s->x32;
    u.r = s->r32;
    u.p = s->p32;
    u.q = s->q32;
    u.st = &b->d_states[s->sidx];
    u.partials = s->partials;
    up.push_back(u);
  }
  std::vector<Launch> L;
  TRYB(prep_operator<float>(b, inner, true, L));
  TRYB(prep_cg<float>(b, CG_PROJECT_DOT, pd, L));
  TRYB(prep_cg<float>(b, CG_UPDATE, up, L));
  TRYB(b->arena.flush(b->stream));
  // The K iterations launch the same kernels on the same work items: capture
  // one iteration as a CUDA graph and replay it K times.
  if (b->graph) {
    GHB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  std::lock_guard<std::mutex> capture_lock(b->capture_mu);
  GHB_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
  ghb_status st = GHB_OK;
  for (const Launch& l : L) {
    st = run_launch(b, l);
    if (st != GHB_OK) break;
  }
  const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
  if (st != GHB_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != GHB_OK) return st;
    GHB_CUDA_TRY(ce);
  }
  const cudaError_t ci = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  GHB_CUDA_TRY(ci);
  for (int it = 0; it < K; ++it) GHB_CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
  b->launches += static_cast<int64_t>(K - 1) * static_cast<int64_t>(L.size());   // run_launch counted one
  return GHB_OK;
}

// FP64 correction of the solves whose inner CG ended.
ghb_status correct(ghb_batch* b) {
  TRYB(read_states(b));
  std::vector<Slot*> ready;
  for (Inst* in : b->active)
    for (int s = 0; s < in->nslots; ++s) {
      Slot& sl = in->slots[s];
      if (sl.state != S_INNER) continue;
      const CgState& st = b->h_states[sl.sidx];
      if (st.done == RUNNING) continue;
      sl.inner_iters += st.iter;
      sl.mv32 += st.iter;
      ready.push_back(&sl);
    }
  if (ready.empty()) return GHB_OK;
  std::vector<CgItem> acc, prj, res, prj2;
  for (Slot* s : ready) {
    CgItem a = cg_item(*s);
    a.x = s->xacc;
    a.w = s->x64;
    a.p = s->x32;
    acc.push_back(a);
    CgItem p = cg_item(*s);
    p.q = s->x64;
    p.w = s->xacc;
    prj.push_back(p);
    CgItem q = cg_item(*s);
    q.q = s->y64;
    q.w = s->w64;
    prj2.push_back(q);
    CgItem r = cg_item(*s);
    r.r = s->r64;
    r.b = s->b64;
    r.w = s->y64;
    r.st = &b->d_states[s->sidx];
    r.partials = s->partials;
    res.push_back(r);
  }
  {
    std::vector<Launch> L;
    TRYB(prep_cg<double>(b, CG_ACCUM, acc, L));       // xacc = x64 + dx
    TRYB(prep_cg<double>(b, CG_PROJECT, prj, L));     // x64 = G xacc (exact, real part)
    TRYB(prep_operator<double>(b, ready, false, L));   // w64 = A^full x64
    TRYB(prep_cg<double>(b, CG_PROJECT, prj2, L));    // y64 = G w64
    TRYB(prep_cg<double>(b, CG_RESIDUAL, res, L));    // r64 = b - y64, <r, r>
    TRYB(run_all(b, L));
  }
  TRYB(read_states(b));
  std::vector<Slot*> again;
  for (Slot* s : ready) {
    s->outer += 1;
    s->mv64 += 1;
    const double rr = b->h_states[s->sidx].rr;
    s->relres = s->bb > 0 ? std::sqrt(rr / s->bb) : 0.0;
    const bool conv = rr <= b->opt.tol * b->opt.tol * s->bb;
    const bool out_of_budget = s->outer >= b->opt.max_outer || s->inner_iters >= b->opt.max_iter;
    if (conv || out_of_budget || !std::isfinite(rr)) {
      s->status = conv ? GHB_OK : (!std::isfinite(rr) ? GHB_ERR_BREAKDOWN : GHB_ERR_NOT_CONVERGED);
      s->state = S_DONE;
      double E[3] = {0, 0, 0};
      E[s->load] = 1.0;
      TRYB(launch_add_constant(s->sol, s->x64, fgeom_of(s->inst->g), E, b->stream));
    } else {
      again.push_back(s);
    }
  }
  return start_inner(b, again);
}

bool inverse_small(int d, const double* A, double* X) {
  if (d == 2) {
    const double det = A[0] * A[3] - A[1] * A[2];
    if (!(det > 0)) return false;
    X[0] = A[3] / det; X[1] = -A[1] / det; X[2] = -A[2] / det; X[3] = A[0] / det;
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

// Gram energies of finished instances (batched), results, memory back to the pool.
ghb_status retire(ghb_batch* b) {
  std::vector<Inst*> fin;
  for (Inst* in : b->active) {
    bool all = true;
    for (int s = 0; s < in->nslots; ++s) all = all && in->slots[s].state == S_DONE;
    if (all) fin.push_back(in);
  }
  if (fin.empty()) return GHB_OK;
  for (int d = 2; d <= 3; ++d) {
    std::vector<ColItem> c1, c2;
    std::vector<int> M0, M1, Md;
    std::vector<RowItem> rw;
    for (Inst* in : fin) {
      if (in->g.d != d) continue;
      const Geometry& g = in->g;
      for (int kind = 0; kind < 2; ++kind) {
        RowItem r{};
        for (int f = 0; f < d; ++f) {
          Slot& s = in->slots[kind * d + f];
          ColItem a{};
          a.a.in = s.sol;
          a.a.out = s.T1_64;
          a.a.outer = d;
          a.a.inner = g.P / g.N[0];
          a.a.Lin = g.N[0];
          a.a.Lout = g.M[0];
          a.pl = in->dpl[0];
          c1.push_back(a);
          M0.push_back(g.M[0]);
          r.a.t[f] = s.T1_64;
          if (d == 3) {
            ColItem c{};
            c.a.in = s.T1_64;
            c.a.out = s.T2_64;
            c.a.outer = static_cast<int64_t>(d) * g.M[0];
            c.a.inner = g.h;
            c.a.Lin = g.N[1];
            c.a.Lout = g.M[1];
            c.pl = in->dpl[1];
            c2.push_back(c);
            M1.push_back(g.M[1]);
            r.a.t[f] = s.T2_64;
          }
        }
        r.a.nfields = d;
        r.a.ncomp = d;
        r.a.rows = g.rows;
        r.a.H = g.h;
        r.a.comp_stride = g.rows * g.h;
        r.a.a = in->grid64[kind];
        r.a.partials = in->gram_partials[kind];
        r.a.gram = in->gram_d + 9 * kind;
        r.a.ticket = in->gram_ticket + kind;
        r.a.scale = 1.0 / static_cast<double>(g.grid);
        r.pl = in->dpl[d - 1];
        rw.push_back(r);
        Md.push_back(g.M[d - 1]);
      }
      GHB_CUDA_TRY(cudaMemsetAsync(in->gram_ticket, 0, 64, b->stream));
    }
    std::vector<Launch> L;
    TRYB(prep_col<double>(b, +1, COL_PLAIN, c1, M0, L));
    TRYB(prep_col<double>(b, +1, COL_PLAIN, c2, M1, L));
    TRYB(prep_row<double>(b, ROW_ENERGY, rw, Md, d, d, L));
    TRYB(run_all(b, L));
  }
  GHB_CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->arena.reset();
  const double t = now_s();
  for (Inst* in : fin) {
    double G[18];
    GHB_CUDA_TRY(cudaMemcpy(G, in->gram_d, sizeof(G), cudaMemcpyDeviceToHost));
    const int d = in->g.d;
    ghb_result r{};
    r.id = in->id;
    r.d = d;
    r.status = GHB_OK;
    double Ds[9], L[9];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        r.upper[i * d + j] = 0.5 * (G[i * d + j] + G[j * d + i]);
        Ds[i * d + j] = 0.5 * (G[9 + i * d + j] + G[9 + j * d + i]);
      }
    if (!inverse_small(d, Ds, L)) r.status = GHB_ERR_BREAKDOWN;
    else
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) r.lower[i * d + j] = 0.5 * (L[i * d + j] + L[j * d + i]);
    for (int s = 0; s < in->nslots; ++s) {
      const Slot& sl = in->slots[s];
      ghb_solve_info& inf = r.info[s];
      inf.status = sl.status;
      inf.iters = sl.inner_iters;
      inf.outer_iters = sl.outer;
      inf.matvecs_fp32 = sl.mv32;
      inf.matvecs_fp64 = sl.mv64;
      inf.relres = sl.relres;
      inf.energy = G[(s < d ? 0 : 9) + (s % d) * d + (s % d)];
      if (sl.status != GHB_OK && r.status == GHB_OK) r.status = sl.status;
      b->free_states.push_back(sl.sidx);
    }
    r.seconds_queued = in->t_admit - in->t_submit;
    r.seconds_total = t - in->t_submit;
    b->results.push_back(r);
    ++b->finished;
    cudaFreeAsync(in->block, b->stream);
    b->in_use -= in->bytes;
  }
  std::vector<Inst*> keep;
  for (Inst* in : b->active)
    if (std::find(fin.begin(), fin.end(), in) == fin.end()) keep.push_back(in);
    else delete in;
  b->active.swap(keep);
  return GHB_OK;
}

}  // namespace

// A large-request worker: one request at a time through a private context.
void lane_main(ghb_batch* b) {
  LargeLane& ln = b->lane;
  cudaSetDevice(ln.device);
  for (;;) {
    Request rq;
    {
      std::unique_lock<std::mutex> lk(ln.mu);
      ln.cv.wait(lk, [&] { return ln.stop || !ln.queue.empty(); });
      if (ln.stop) return;
      rq = std::move(ln.queue.front());
      ln.queue.pop_front();
      ++ln.running;
    }
    ghb_result r{};
    r.id = rq.id;
    r.d = rq.d;
    const double t_start = now_s();
    ghb_ctx* c = nullptr;
    ghb_status st;
    {
      std::lock_guard<std::mutex> g(b->capture_mu);
      st = ghb_create(&c, rq.d, rq.N, rq.a0, rq.phases.empty() ? nullptr : rq.phases.data(),
                      static_cast<int>(rq.phases.size()), &b->opt);
    }
    if (st == GHB_OK) {
      const int64_t bytes = ghb_device_bytes(c);
      b->in_use += bytes;
      st = ghb_bounds(c, r.upper, r.lower, r.info);
      {
        std::lock_guard<std::mutex> g(b->capture_mu);
        ghb_destroy(c);
      }
      b->in_use -= bytes;
    }
    r.status = st;
    r.seconds_queued = t_start - rq.t_submit;
    r.seconds_total = now_s() - rq.t_submit;
    {
      std::lock_guard<std::mutex> lk(ln.mu);
      ln.done.push_back(r);
      --ln.running;
    }
    ln.cv.notify_all();
  }
}

// Results of the worker into the batch's queue; with `wait`, block up to 50 ms
// for one while the worker is busy.
void drain_lane(ghb_batch* b, bool wait) {
  LargeLane& ln = b->lane;
  std::unique_lock<std::mutex> lk(ln.mu);
  if (wait && ln.done.empty() && (ln.running || !ln.queue.empty()))
    ln.cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return !ln.done.empty(); });
  while (!ln.done.empty()) {
    b->results.push_back(ln.done.front());
    ln.done.pop_front();
    ++b->finished;
  }
}

bool lane_busy(ghb_batch* b) {
  std::lock_guard<std::mutex> lk(b->lane.mu);
  return b->lane.running || !b->lane.queue.empty() || !b->lane.done.empty();
}

extern "C" {

ghb_status ghb_batch_create(ghb_batch** out, const ghb_options* opt, int64_t budget_bytes, int max_active) {
  clear_error();
  if (!out) { set_error("out is NULL"); return GHB_ERR_INVALID; }
  *out = nullptr;
  ghb_options o;
  ghb_default_options(&o);
  o.precision = GHB_MIXED;
  if (opt) o = *opt;
  if (o.precision != GHB_MIXED) {
    set_error("the batch engine runs the mixed scheme (FP32 inner CG, FP64 correction)");
    return GHB_ERR_INVALID;
  }
  if (!(o.tol > 0 && o.tol < 1) || !(o.inner_tol > 0 && o.inner_tol < 1) || o.max_iter < 1 || o.max_outer < 1) {
    set_error("invalid options");
    return GHB_ERR_INVALID;
  }
  ghb_batch* b = new ghb_batch();
  b->opt = o;
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    delete b;
    return GHB_ERR_CUDA;
  }
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  b->budget = budget_bytes > 0 ? budget_bytes : static_cast<int64_t>(0.6 * static_cast<double>(fr));
  b->max_active = max_active > 0 ? max_active : 4096;
  // keep freed instance blocks in the pool for the next admissions
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  b->cap_states = 6 * b->max_active;
  if (cudaMalloc(&b->d_states, sizeof(CgState) * b->cap_states) != cudaSuccess ||
      cudaMallocHost(&b->h_states, sizeof(CgState) * b->cap_states) != cudaSuccess) {
    set_error("state allocation failed");
    ghb_batch_destroy(b);
    return GHB_ERR_OOM;
  }
  cudaMemset(b->d_states, 0, sizeof(CgState) * b->cap_states);
  if (b->arena.init(static_cast<size_t>(64) << 20) != GHB_OK) {
    ghb_batch_destroy(b);
    return GHB_ERR_OOM;
  }
  for (int i = b->cap_states - 1; i >= 0; --i) b->free_states.push_back(i);
  *out = b;
  return GHB_OK;
}

ghb_status ghb_batch_submit(ghb_batch* b, int d, const int* N, double a0, const ghb_phase* phases, int n_phases,
                            int64_t* id_out) {
  clear_error();
  if (!b || !N) { set_error("null argument"); return GHB_ERR_INVALID; }
  if (d != 2 && d != 3) { set_error("d must be 2 or 3"); return GHB_ERR_INVALID; }
  Geometry g;
  TRYB(make_geometry(d, N, b->opt, &g));
  if (!(a0 > 0) || n_phases < 0 || (n_phases > 0 && !phases)) { set_error("invalid microstructure"); return GHB_ERR_INVALID; }
  for (int i = 0; i < n_phases; ++i) {
    const ghb_phase& p = phases[i];
    const bool round = (p.shape == GHB_DISK && d == 2) || (p.shape == GHB_SPHERE && d == 3);
    if (!(p.value > 0) || !(round || p.shape == GHB_BOX)) { set_error("invalid inclusion"); return GHB_ERR_INVALID; }
    if (round && !(p.size[0] > 0 && p.size[0] <= 0.5)) { set_error("radius must lie in (0, 1/2]"); return GHB_ERR_INVALID; }
    if (!round)
      for (int a = 0; a < d; ++a)
        if (!(p.size[a] > 0 && p.size[a] <= 1)) { set_error("box sides must lie in (0, 1]"); return GHB_ERR_INVALID; }
  }
  Request r;
  r.id = b->next_id++;
  r.d = d;
  for (int a = 0; a < 3; ++a) r.N[a] = a < d ? N[a] : 1;
  r.a0 = a0;
  r.phases.assign(phases, phases + n_phases);
  r.t_submit = now_s();
  if (id_out) *id_out = r.id;
  if (g.grid >= kLargeGrid) {
    LargeLane& ln = b->lane;
    if (ln.workers.empty()) {
      cudaGetDevice(&ln.device);
      for (int w = 0; w < kLaneWorkers; ++w) ln.workers.emplace_back(lane_main, b);
    }
    {
      std::lock_guard<std::mutex> lk(ln.mu);
      ln.queue.push_back(std::move(r));
    }
    ln.cv.notify_all();
    return GHB_OK;
  }
  b->pending.push_back(r);
  return GHB_OK;
}

ghb_status ghb_batch_step(ghb_batch* b, int iterations, int* active_out, int* pending_out) {
  clear_error();
  if (!b) { set_error("batch is NULL"); return GHB_ERR_INVALID; }
  try {
    TRYB(admit(b));
    TRYB(iterate(b, iterations > 0 ? iterations : 8));
    TRYB(correct(b));
    TRYB(retire(b));
    // with no batched work left, wait briefly for the large-request worker
    // instead of returning at once to a caller that loops on ghb_batch_step
    drain_lane(b, b->active.empty() && b->pending.empty());
  } catch (const std::exception& ex) {
    set_error(std::string("internal error: ") + ex.what());
    return GHB_ERR_INVALID;
  }
  int lane_active = 0, lane_pending = 0;
  {
    std::lock_guard<std::mutex> lk(b->lane.mu);
    lane_active = b->lane.running;
    lane_pending = static_cast<int>(b->lane.queue.size());
  }
  if (active_out) *active_out = static_cast<int>(b->active.size()) + lane_active;
  if (pending_out) *pending_out = static_cast<int>(b->pending.size()) + lane_pending;
  return GHB_OK;
}

ghb_status ghb_batch_run(ghb_batch* b, int iterations) {
  if (!b) { set_error("batch is NULL"); return GHB_ERR_INVALID; }
  while (!b->active.empty() || !b->pending.empty() || lane_busy(b))
    TRYB(ghb_batch_step(b, iterations, nullptr, nullptr));
  return GHB_OK;
}

int ghb_batch_results(ghb_batch* b, ghb_result* out, int max_results) {
  if (!b || !out) return 0;
  int n = 0;
  while (n < max_results && !b->results.empty()) {
    out[n++] = b->results.front();
    b->results.pop_front();
  }
  return n;
}

ghb_status ghb_batch_stats(const ghb_batch* b, int64_t* bytes_in_use, int* active, int* pending,
                           int64_t* finished, int64_t* launches) {
  if (!b) { set_error("batch is NULL"); return GHB_ERR_INVALID; }
  LargeLane& ln = const_cast<ghb_batch*>(b)->lane;
  int lane_active = 0, lane_pending = 0;
  {
    std::lock_guard<std::mutex> lk(ln.mu);
    lane_active = ln.running;
    lane_pending = static_cast<int>(ln.queue.size());
  }
  if (bytes_in_use) *bytes_in_use = b->in_use;
  if (active) *active = static_cast<int>(b->active.size()) + lane_active;
  if (pending) *pending = static_cast<int>(b->pending.size()) + lane_pending;
  if (finished) *finished = b->finished;
  if (launches) *launches = b->launches;
  return GHB_OK;
}

void ghb_batch_destroy(ghb_batch* b) {
  if (!b) return;
  if (!b->lane.workers.empty()) {   // requests in progress finish; queued ones are dropped
    {
      std::lock_guard<std::mutex> lk(b->lane.mu);
      b->lane.stop = true;
      b->lane.queue.clear();
    }
    b->lane.cv.notify_all();
    for (auto& w : b->lane.workers) w.join();
  }
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (Inst* in : b->active) {
    if (in->block) cudaFreeAsync(in->block, b->stream);
    delete in;
  }
  for (auto& kv : b->plans) {
    free_plan(kv.second.h);
    if (kv.second.d_plan) cudaFree(kv.second.d_plan);
  }
  b->arena.release();
  if (b->d_states) cudaFree(b->d_states);
  if (b->h_states) cudaFreeHost(b->h_states);
  if (b->stream) {
    cudaStreamSynchronize(b->stream);
    cudaStreamDestroy(b->stream);
  }
  delete b;
}

}  // extern "C"
