// Autotuner of the operator's launch configuration, per transform length M.
//
// What it chooses (carried in every FftPlan made for M):
//   cap32, cap64  largest radix product of a register-blocked pass of the
//                 runtime-plan transform (FP32, FP64): fewer passes against
//                 more registers per thread;
//   rows32        rows per CTA of the FP32 2-D operator's last-axis pass;
//   ct_col/ct_row size-specialised FP32 kernels (where compiled) or the
//                 runtime-plan ones.
// The columns per CTA of the column passes (tile32/64) depend on the operand,
// not on M alone (a 3-D axis-1 pass has ~M times the columns of a 2-D one), so
// they are chosen at launch from the operand's shape (auto_tile) and are not
// tuned; ghb_tune_set can still force them.
// How: on the first plan for M in the process, a 2-D operand with the largest
// odd N that M serves is allocated -- at least 2^20 double-grid entries per
// component, widened with more columns and rows where N x N is smaller, so
// that the timed launches are long enough to compare -- and every candidate is
// timed with CUDA events on a private stream (1 untimed + 3 timed launches;
// the inverse and forward column passes and the last-axis pass separately);
// the fastest runtime-plan grouping by the sum of the three, then the
// specialised kernels where they beat it.  Results stay for the life of the
// process.
// GHB_AUTOTUNE=0 in the environment keeps the size rules instead.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "ghb_internal.cuh"

namespace ghb {
void clear_error();
}  // namespace ghb

using namespace ghb;

namespace {

struct Tune {
  int cap32, tile32, rows32, ct_col, ct_row, cap64, tile64;
};
constexpr int kTuneFields = 7;

std::mutex g_mutex;
std::map<int, Tune> g_tunes;

bool tuning_enabled() {
  const char* e = std::getenv("GHB_AUTOTUNE");
  return !(e != nullptr && e[0] == '0');
}

Tune size_rules(int M) {
  const int ct = ct_size(M) ? 1 : 0;
  return Tune{32, 0, 0, ct, ct, 18, 0};
}

void write_tune(const Tune& t, FftPlan& p) {
  group_passes(p, 1, t.cap32);
  group_passes(p, 0, t.cap64);
  p.tile[1] = t.tile32;
  p.tile[0] = t.tile64;
  p.rows32 = t.rows32;
  const bool ct = p.perm_ct != nullptr && ct_size(p.M);
  p.ct_col = ct ? t.ct_col : 0;
  p.ct_row = ct ? t.ct_row : 0;
}

struct Timer {
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ghb_status init() {
    GHB_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    GHB_CUDA_TRY(cudaEventCreate(&e0));
    GHB_CUDA_TRY(cudaEventCreate(&e1));
    return GHB_OK;
  }
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
  }
  // mean milliseconds of one launch of fn (1 untimed, 3 timed)
  template <typename F>
  ghb_status time(F&& fn, float* ms) {
    {
      const ghb_status st = fn();
      if (st != GHB_OK) return st;
    }
    GHB_CUDA_TRY(cudaEventRecord(e0, s));
    for (int i = 0; i < 3; ++i) {
      const ghb_status st = fn();
      if (st != GHB_OK) return st;
    }
    GHB_CUDA_TRY(cudaEventRecord(e1, s));
    GHB_CUDA_TRY(cudaEventSynchronize(e1));
    float t = 0;
    GHB_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
    *ms = t / 3;
    return GHB_OK;
  }
};

// Scratch of the timing runs, kept for the process and grown when a larger
// length comes (releasing it would synchronise the whole device, stalling
// work that other streams have in flight).
struct Scratch {
  void* p[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t bytes[6] = {0, 0, 0, 0, 0, 0};
  int device = -1;
};
Scratch g_scratch;

ghb_status scratch(int i, size_t bytes, void** out) {
  int dev = 0;
  GHB_CUDA_TRY(cudaGetDevice(&dev));
  if (g_scratch.device != dev) {   // another device: start over (the old buffers stay with it)
    g_scratch = Scratch{};
    g_scratch.device = dev;
  }
  if (g_scratch.bytes[i] < bytes) {
    if (g_scratch.p[i]) cudaFree(g_scratch.p[i]);
    g_scratch.p[i] = nullptr;
    g_scratch.bytes[i] = 0;
    GHB_CUDA_TRY(cudaMalloc(&g_scratch.p[i], bytes));
    g_scratch.bytes[i] = bytes;
  }
  *out = g_scratch.p[i];
  return GHB_OK;
}

#define TUNE_TRY(x)                      \
  do {                                   \
    const ghb_status st_ = (x);          \
    if (st_ != GHB_OK) return st_;       \
  } while (0)

// Times the candidates for length M on a square 2-D operand.
ghb_status tune_length(int M, Tune* out) {
  Tune best = size_rules(M);
  int N = (M + 1) / 2;
  if (N % 2 == 0) --N;
  if (N < 1) {
    *out = best;
    return GHB_OK;
  }
  const int h = (N + 1) / 2;
  // the plan's device tables stay for the process (see Scratch)
  static std::map<std::pair<int, int>, PlanHolder> plans;
  int dev = 0;
  GHB_CUDA_TRY(cudaGetDevice(&dev));
  auto key = std::make_pair(dev, M);
  if (!plans.count(key)) {
    PlanHolder fresh;
    TUNE_TRY(make_plan_untuned(M, fresh));
    plans[key] = fresh;
  }
  const PlanHolder& ph = plans[key];
  Timer tm;
  TUNE_TRY(tm.init());
  struct {
    void* p[6];
  } b;
  // columns of the column passes and rows of the last-axis pass: M and h at
  // least, 2^22 / M where that is more (cols x M >= rows x h always holds, so
  // the last-axis pass's operand fits in the column passes' output)
  constexpr int64_t kTarget = int64_t(1) << 20;
  const int64_t cols = std::max<int64_t>(h, (kTarget + M - 1) / M);
  const int64_t rows = std::max<int64_t>(M, (kTarget + M - 1) / M);
  const size_t nx = 2ull * N * cols, nt = 2ull * M * cols, ng = static_cast<size_t>(rows) * M;
  const size_t sz[6] = {nx * sizeof(float2), nt * sizeof(float2), ng * sizeof(float),
                        nx * sizeof(double2), nt * sizeof(double2), ng * sizeof(double)};
  for (int i = 0; i < 6; ++i) TUNE_TRY(scratch(i, sz[i], &b.p[i]));
  GHB_CUDA_TRY(cudaMemsetAsync(b.p[0], 0, nx * sizeof(float2), tm.s));
  GHB_CUDA_TRY(cudaMemsetAsync(b.p[1], 0, nt * sizeof(float2), tm.s));
  GHB_CUDA_TRY(cudaMemsetAsync(b.p[2], 0, ng * sizeof(float), tm.s));
  GHB_CUDA_TRY(cudaMemsetAsync(b.p[3], 0, nx * sizeof(double2), tm.s));
  GHB_CUDA_TRY(cudaMemsetAsync(b.p[4], 0, nt * sizeof(double2), tm.s));
  GHB_CUDA_TRY(cudaMemsetAsync(b.p[5], 0, ng * sizeof(double), tm.s));

  auto args = [&](bool f32, ColArgs& inv, ColArgs& fwd, RowArgs& row) {
    void* X = b.p[f32 ? 0 : 3];
    void* T1 = b.p[f32 ? 1 : 4];
    inv = ColArgs{};
    inv.in = X;
    inv.out = T1;
    inv.outer = 2;
    inv.inner = cols;
    inv.Lin = N;
    inv.Lout = M;
    fwd = inv;
    fwd.in = T1;
    fwd.out = X;
    fwd.Lin = M;
    fwd.Lout = N;
    row = RowArgs{};
    row.t[0] = T1;
    row.nfields = 1;
    row.ncomp = 2;
    row.rows = rows;
    row.H = h;
    row.comp_stride = rows * h;
    row.a = b.p[f32 ? 2 : 5];
  };

  // FP32: runtime-plan grouping and rows, then the specialised kernels
  {
    ColArgs inv, fwd;
    RowArgs row;
    args(true, inv, fwd, row);
    float best_total = 1e30f, best_col_generic = 1e30f, best_row_generic = 1e30f;
    for (int cap : {18, 32}) {
      FftPlan p = ph.plan;
      group_passes(p, 1, cap);
      p.ct_col = p.ct_row = 0;
      float col_best = 1e30f, row_best = 1e30f;
      int rows_best = 0;
      {
        p.tile[1] = 0;
        float ti = 0, tf = 0;
        TUNE_TRY(tm.time([&] { return launch_col<float>(+1, COL_PLAIN, inv, p, tm.s); }, &ti));
        TUNE_TRY(tm.time([&] { return launch_col<float>(-1, COL_PLAIN, fwd, p, tm.s); }, &tf));
        col_best = ti + tf;
      }
      for (int rows : {1, 2}) {
        p.rows32 = rows;
        float tr = 0;
        TUNE_TRY(tm.time([&] { return launch_row<float>(ROW_MATVEC, row, p, tm.s); }, &tr));
        if (tr < row_best) {
          row_best = tr;
          rows_best = rows;
        }
      }
      if (col_best + row_best < best_total) {
        best_total = col_best + row_best;
        best_col_generic = col_best;
        best_row_generic = row_best;
        best.cap32 = cap;
        best.tile32 = 0;
        best.rows32 = rows_best;
      }
    }
    best.ct_col = best.ct_row = 0;
    if (ph.plan.perm_ct != nullptr && ct_size(M)) {
      FftPlan p = ph.plan;
      p.ct_col = p.ct_row = 1;
      float ti = 0, tf = 0;
      TUNE_TRY(tm.time([&] { return launch_col<float>(+1, COL_PLAIN, inv, p, tm.s); }, &ti));
      TUNE_TRY(tm.time([&] { return launch_col<float>(-1, COL_PLAIN, fwd, p, tm.s); }, &tf));
      if (ti + tf < best_col_generic) best.ct_col = 1;
      for (int rows : {1, 2}) {
        p.rows32 = rows;
        float tr = 0;
        TUNE_TRY(tm.time([&] { return launch_row<float>(ROW_MATVEC, row, p, tm.s); }, &tr));
        if (tr < best_row_generic) {
          best_row_generic = tr;
          best.ct_row = 1;
          best.rows32 = rows;
        }
      }
    }
  }
  // FP64: grouping (the last-axis pass at one row per CTA)
  {
    ColArgs inv, fwd;
    RowArgs row;
    args(false, inv, fwd, row);
    float best_total = 1e30f;
    for (int cap : {9, 18}) {
      FftPlan p = ph.plan;
      group_passes(p, 0, cap);
      float col_best = 1e30f;
      {
        p.tile[0] = 0;
        float ti = 0, tf = 0;
        TUNE_TRY(tm.time([&] { return launch_col<double>(+1, COL_PLAIN, inv, p, tm.s); }, &ti));
        TUNE_TRY(tm.time([&] { return launch_col<double>(-1, COL_PLAIN, fwd, p, tm.s); }, &tf));
        col_best = ti + tf;
      }
      float tr = 0;
      TUNE_TRY(tm.time([&] { return launch_row<double>(ROW_MATVEC, row, p, tm.s); }, &tr));
      if (col_best + tr < best_total) {
        best_total = col_best + tr;
        best.cap64 = cap;
        best.tile64 = 0;
      }
    }
  }
  *out = best;
  return GHB_OK;
}

bool valid_tune(int M, const Tune& t) {
  const bool caps = t.cap32 >= 5 && t.cap32 <= 32 && t.cap64 >= 5 && t.cap64 <= 32;
  auto tile_ok = [&](int tile, int eb) {
    return tile == 0 || ((tile == 1 || tile == 2 || tile == 4 || tile == 8 || tile == 16) &&
                         col_smem_bytes(M, tile, eb) <= 220 * 1024);
  };
  const bool rows = t.rows32 >= 0 && t.rows32 <= 2;
  const bool ct = (t.ct_col == 0 || t.ct_col == 1) && (t.ct_row == 0 || t.ct_row == 1) &&
                  (ct_size(M) || (t.ct_col == 0 && t.ct_row == 0));
  return caps && tile_ok(t.tile32, 8) && tile_ok(t.tile64, 16) && rows && ct;
}

// The configuration for M: stored, else tuned (if enabled), else the size rules.
ghb_status tune_of(int M, Tune* out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  auto it = g_tunes.find(M);
  if (it != g_tunes.end()) {
    *out = it->second;
    return GHB_OK;
  }
  Tune t = size_rules(M);
  if (tuning_enabled()) {
    const ghb_status st = tune_length(M, &t);
    if (st != GHB_OK) return st;
  }
  g_tunes[M] = t;
  *out = t;
  return GHB_OK;
}

}  // namespace

namespace ghb {

ghb_status apply_tune(int M, FftPlan& p) {
  Tune t{};
  const ghb_status st = tune_of(M, &t);
  if (st != GHB_OK) return st;
  write_tune(t, p);
  return GHB_OK;
}

}  // namespace ghb

extern "C" {

ghb_status ghb_tune_get(int M, int* cfg) {
  clear_error();
  if (cfg == nullptr || M < 1 || !factorizable(M)) {
    set_error("ghb_tune_get: M must factor into primes <= 31 and cfg must not be NULL");
    return GHB_ERR_INVALID;
  }
  Tune t{};
  const ghb_status st = tune_of(M, &t);
  if (st != GHB_OK) return st;
  const int v[kTuneFields] = {t.cap32, t.tile32, t.rows32, t.ct_col, t.ct_row, t.cap64, t.tile64};
  std::memcpy(cfg, v, sizeof(v));
  return GHB_OK;
}

ghb_status ghb_tune_set(int M, const int* cfg) {
  clear_error();
  if (cfg == nullptr || M < 1 || !factorizable(M)) {
    set_error("ghb_tune_set: M must factor into primes <= 31 and cfg must not be NULL");
    return GHB_ERR_INVALID;
  }
  const Tune t{cfg[0], cfg[1], cfg[2], cfg[3], cfg[4], cfg[5], cfg[6]};
  if (!valid_tune(M, t)) {
    set_error("ghb_tune_set: invalid configuration (caps 5..32, tiles 0/1/2/4/8/16 within shared memory, "
              "rows 0..2, specialised kernels 0/1 and only for lengths that have them)");
    return GHB_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  g_tunes[M] = t;
  return GHB_OK;
}

ghb_status ghb_tune_reset(void) {
  clear_error();
  std::lock_guard<std::mutex> lock(g_mutex);
  g_tunes.clear();
  return GHB_OK;
}

}  // extern "C"
