// ghb_gram_noalloc: the Gram energies of ghb_gram without any device
// allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- code that runs inside
// another framework's memory arena or pool and must not grow the device heap
// behind its back, code that runs while device memory is reserved to the last
// byte, or code under a policy that forbids allocation after start-up.  They
// pass their own inputs and outputs; everything else this computation needs
// (transform tables, the intermediates of the padded inverse transforms, the
// per-block partial sums and the Gram matrix) lives in one file-scope device
// array of kNoAllocScratchBytes below, which every GPU that loads this library
// holds until the process exits.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ghb_internal.cuh"

namespace ghb {
void clear_error();
}  // namespace ghb

using namespace ghb;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is a host-side stand-in, not a
// device address: host code obtains the address with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
ghb_status scratch_address(unsigned char** out) {
  int dev = 0;
  GHB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index out of range for the no-allocation scratch");
    return GHB_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
      return GHB_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return GHB_OK;
}

size_t al256(size_t n) { return (n + 255) & ~static_cast<size_t>(255); }

}  // namespace

extern "C" {

ghb_status ghb_gram_noalloc(int d, const int* N, const int* M, const double* grid_dev, int m,
                            const void* const* fields_dev, double* out, void* stream) {
  clear_error();
  if ((d != 2 && d != 3) || !N || !M || !grid_dev || !fields_dev || !out) {
    set_error("ghb_gram_noalloc: d must be 2 or 3 and no pointer may be NULL");
    return GHB_ERR_INVALID;
  }
  if (m < 1 || m > d) {
    set_error("ghb_gram_noalloc: m must lie in 1..d");
    return GHB_ERR_INVALID;
  }
  for (int i = 0; i < m; ++i)
    if (!fields_dev[i]) {
      set_error("ghb_gram_noalloc: null field");
      return GHB_ERR_INVALID;
    }
  Geometry g{};
  g.d = d;
  for (int a = 0; a < 3; ++a) { g.N[a] = 1; g.M[a] = 1; }
  for (int a = 0; a < d; ++a) {
    if (N[a] < 1 || N[a] % 2 == 0 || M[a] < 2 * N[a] - 1 || !factorizable(M[a])) {
      set_error("ghb_gram_noalloc: N must be odd and M >= 2N - 1 with prime factors <= 31");
      return GHB_ERR_INVALID;
    }
    g.N[a] = N[a];
    g.M[a] = M[a];
  }
  g.h = (g.N[d - 1] + 1) / 2;
  g.P = g.h;
  for (int a = 0; a < d - 1; ++a) g.P *= g.N[a];
  g.T1 = static_cast<int64_t>(d) * g.M[0] * (g.P / g.N[0]);
  g.T2 = d == 3 ? static_cast<int64_t>(d) * g.M[0] * g.M[1] * g.h : 0;
  g.rows = d == 2 ? g.M[0] : static_cast<int64_t>(g.M[0]) * g.M[1];
  g.grid = 1;
  for (int a = 0; a < d; ++a) g.grid *= g.M[a];
  const int Md = g.M[d - 1];
  const int NL = (m * d + 1) / 2;   // interleaved complex lines of the Gram pass
  if (padded_elems<double2>(static_cast<size_t>(NL) * Md) * sizeof(double2) > 200 * 1024) {
    set_error("ghb_gram_noalloc: M too large for one CTA's shared memory");
    return GHB_ERR_INVALID;
  }

  // plans (distinct M share one) and their tables
  FftPlan pl[3];
  PlanTables tab[3];
  int plan_of[3] = {0, 1, 2};
  for (int a = 0; a < d; ++a) {
    plan_of[a] = a;
    for (int b = 0; b < a; ++b)
      if (g.M[b] == g.M[a]) plan_of[a] = plan_of[b];
    if (plan_of[a] == a) {
      const ghb_status st = build_plan_tables(g.M[a], pl[a], tab[a]);
      if (st != GHB_OK) return st;
    }
  }

  // scratch layout: tables, intermediates, partial sums, ticket, Gram
  size_t need = 0;
  size_t off_tab[3][3] = {{0}};
  for (int a = 0; a < d; ++a) {
    if (plan_of[a] != a) continue;
    const size_t sz[3] = {sizeof(int) * tab[a].perm.size(), sizeof(double2) * tab[a].tw64.size(),
                          sizeof(float2) * tab[a].tw32.size()};
    for (int k = 0; k < 3; ++k) {
      off_tab[a][k] = need;
      need += al256(sz[k]);
    }
  }
  size_t off_T1[3], off_T2[3];
  for (int f = 0; f < m; ++f) {
    off_T1[f] = need;
    need += al256(sizeof(double2) * g.T1);
    off_T2[f] = need;
    need += al256(sizeof(double2) * (d == 3 ? g.T2 : 1));
  }
  const size_t off_part = need;
  need += al256(sizeof(double) * 1024 * 6);
  const size_t off_ticket = need;
  need += 256;
  const size_t off_gram = need;
  need += 256;
  if (need > kNoAllocScratchBytes) {
    set_error("ghb_gram_noalloc: these sizes need " + std::to_string(need) +
              " bytes of scratch, more than the fixed " + std::to_string(kNoAllocScratchBytes) +
              " (use ghb_gram, which allocates)");
    return GHB_ERR_INVALID;
  }

  unsigned char* base = nullptr;
  {
    const ghb_status st = scratch_address(&base);
    if (st != GHB_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // tables into the scratch (pageable host sources: each copy is staged
  // before the call returns, so the host vectors may go out of scope)
  for (int a = 0; a < d; ++a) {
    if (plan_of[a] != a) continue;
    GHB_CUDA_TRY(cudaMemcpyAsync(base + off_tab[a][0], tab[a].perm.data(), sizeof(int) * tab[a].perm.size(),
                                 cudaMemcpyHostToDevice, s));
    GHB_CUDA_TRY(cudaMemcpyAsync(base + off_tab[a][1], tab[a].tw64.data(), sizeof(double2) * tab[a].tw64.size(),
                                 cudaMemcpyHostToDevice, s));
    GHB_CUDA_TRY(cudaMemcpyAsync(base + off_tab[a][2], tab[a].tw32.data(), sizeof(float2) * tab[a].tw32.size(),
                                 cudaMemcpyHostToDevice, s));
    pl[a].perm = reinterpret_cast<const int*>(base + off_tab[a][0]);
    pl[a].tw64 = reinterpret_cast<const double2*>(base + off_tab[a][1]);
    pl[a].tw32 = reinterpret_cast<const float2*>(base + off_tab[a][2]);
  }
  // the Gram pass's completion counter must start at zero on every call
  GHB_CUDA_TRY(cudaMemsetAsync(base + off_ticket, 0, 256, s));

  RowArgs r{};
  for (int f = 0; f < m; ++f) {
    double2* T1 = reinterpret_cast<double2*>(base + off_T1[f]);
    double2* T2 = reinterpret_cast<double2*>(base + off_T2[f]);
    ColArgs a{};
    a.in = fields_dev[f];
    a.out = T1;
    a.outer = d;
    a.inner = g.P / g.N[0];
    a.Lin = g.N[0];
    a.Lout = g.M[0];
    {
      const ghb_status st = launch_col<double>(+1, COL_PLAIN, a, pl[plan_of[0]], s);
      if (st != GHB_OK) return st;
    }
    r.t[f] = T1;
    if (d == 3) {
      ColArgs b{};
      b.in = T1;
      b.out = T2;
      b.outer = static_cast<int64_t>(d) * g.M[0];
      b.inner = g.h;
      b.Lin = g.N[1];
      b.Lout = g.M[1];
      const ghb_status st = launch_col<double>(+1, COL_PLAIN, b, pl[plan_of[1]], s);
      if (st != GHB_OK) return st;
      r.t[f] = T2;
    }
  }
  r.nfields = m;
  r.ncomp = d;
  r.rows = g.rows;
  r.H = g.h;
  r.comp_stride = g.rows * g.h;
  r.a = grid_dev;
  r.partials = reinterpret_cast<double*>(base + off_part);
  r.gram = reinterpret_cast<double*>(base + off_gram);
  r.ticket = reinterpret_cast<unsigned int*>(base + off_ticket);
  r.scale = 1.0 / static_cast<double>(g.grid);
  {
    const ghb_status st = launch_row<double>(ROW_ENERGY, r, pl[plan_of[d - 1]], s);
    if (st != GHB_OK) return st;
  }
  double h[9];
  GHB_CUDA_TRY(cudaMemcpyAsync(h, base + off_gram, sizeof(double) * m * m, cudaMemcpyDeviceToHost, s));
  GHB_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < m * m; ++i) out[i] = h[i];
  return GHB_OK;
}

}  // extern "C"
