// Kernel templates of the transform passes of the double-grid Ga operator (Algorithm 2 on the Fourier
// side, Cor. Ga_linsys; Lemma integ_eval_VM):
//
//   column pass  -- zero-pad Z_N -> Z_M and inverse DFT (or forward DFT and
//                   truncate Z_M -> Z_N) along one non-contiguous axis, for a
//                   tile of TW neighbouring lines held interleaved in shared
//                   memory (rows of TW contiguous entries are read and written);
//   row pass     -- the contiguous last axis, stored as a half spectrum:
//                   Hermitian completion, inverse DFT to real values, then
//                     MATVEC: multiply by A_M(x_m) and transform back,
//                     TOREAL: store the real values (the double-grid values
//                             A_M of eq. MBA_GA),
//                     ENERGY: accumulate the Gram sums
//                             (1/|M|) sum_m A_M(x_m) v_i(x_m).v_j(x_m).
//                   Two real lines share one complex transform (z = u + i v).
//
// The templates are instantiated in several translation units (one per
// precision and tile-width group) so that the library compiles in parallel.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "fft_ct.cuh"
#include "ghb_internal.cuh"
#include "reduce.cuh"

namespace ghb {

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async): every thread issues its
// copies back to back and waits once, so a CTA's loads are all in flight
// together instead of one dependent load per loop iteration.
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst_smem, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The dynamic shared-memory limit of kernel `func` raised to `bytes` on the
// current device.  The attribute belongs to the device's context, so it is set
// once per device (bit `dev` of `mask`, one mask per kernel); two host threads
// may both set it, which is harmless.  Devices beyond 63 set it every time.
template <typename F>
inline ghb_status ensure_dyn_smem(F* func, int bytes, std::atomic<unsigned long long>& mask) {
  int dev = 0;
  GHB_CUDA_TRY(cudaGetDevice(&dev));
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit == 0 || !(mask.load(std::memory_order_acquire) & bit)) {
    GHB_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    mask.fetch_or(bit, std::memory_order_release);
  }
  return GHB_OK;
}

// Shared-memory index of entry i: padded for the runtime-plan transform,
// plain for the size-specialised one (MCT = its compile-time length).
template <int MCT, typename C>
__device__ __forceinline__ int bix(int i) {
  if constexpr (MCT != 0) return i;
  else return pidx<C>(i);
}

// Butterflies of one line in the pass with the fewest (the size-specialised
// plan of length M): a CTA of the last-axis pass keeps all its threads busy
// only if its interleaved lines times this count reach its thread count.
template <int M>
__host__ __device__ constexpr int ct_min_units() {
  constexpr CtPlan P = ct_plan(M);
  int mn = M;
  for (int i = 0; i < P.npass; ++i) {
    const int u = M / (P.ra[i] * P.rb[i] * P.rc[i]);
    if (u < mn) mn = u;
  }
  return mn;
}
// Threads of a column-pass CTA.  Runtime plans: 512 (FP32) or 256 (FP64).
// Size-specialised transforms: one thread per butterfly of the pass with the
// fewest (TW lines of ct_min_units each), in whole warps, between 128 and 672
// (FP32) or 352 (FP64) -- FP64 holds a radix group of up to 27 complex
// doubles per thread, which needs more than the 128 registers a 512-thread
// CTA allows.  At M = 4374 the 4 x 162 FP32 (2 x 162 FP64) radix-27
// butterflies of a tile take one round of 672 (352) threads instead of two
// rounds of 512 (256), the second about a quarter full: FP32 axis-1 inverse
// 68 -> 60 us, forward 64 -> 61 us; FP64 1.20 -> 1.15 ms each.  672 threads
// leave 80 registers, which the FP32 inverse pass with the p update exceeds
// (it spilled and measured 89 against 86 us), so the p-update variants keep
// 512 (256).  col_min_blocks keeps the register budget of a full block.
template <typename T, int TW, int MCT, int MODE = COL_PLAIN>
__host__ __device__ constexpr int col_threads() {
  if constexpr (MCT != 0) {
    constexpr int full = sizeof(T) == 4 ? (MODE == COL_PUPDATE ? 512 : 672) : (MODE == COL_PUPDATE ? 256 : 352);
    int t = ((ct_min_units<MCT>() * TW + 31) / 32) * 32;
    if (t < 128) t = 128;
    return t < full ? t : full;
  } else {
    return sizeof(T) == 8 ? 256 : 512;
  }
}
// Resident blocks the compiler must allow for: as many as make up a full
// block's threads; FP32 one fewer when that leaves fewer than the 96
// registers a radix-27 group needs (448 threads at M = 1458 were held to 72
// registers by two blocks and spilled 208 bytes: p-update inverse pass
// 19.4 -> 17.0 us).  (FP64 at M = 1458 measured 3 % slower with one block.)
template <typename T, int TW, int MCT, int MODE = COL_PLAIN>
__host__ __device__ constexpr int col_min_blocks() {
  constexpr int full = sizeof(T) == 4 ? 512 : 256;
  constexpr int t = col_threads<T, TW, MCT, MODE>();
  constexpr int need = sizeof(T) == 4 ? 96 : 0;
  int b = (full + t - 1) / t;
  if (b > 1 && 65536 / (b * t) < need) --b;
  return b;
}

// ---------------------------------------------------------------------------
// column pass: block `bid` of one operand handles tile (o, j0..j0+TW)
// ---------------------------------------------------------------------------
// Input of the size-specialised inverse column transform: entry n of tile
// line t is input row i(n) = n + half (n <= half) or n - M + half
// (n >= M - half), zero in between; with UPDATE the entry is r + beta p_old
// and is written back to p_new once all of a unit's entries are loaded.
// off[t] is the element offset of row 0 of line t's column (a tile's lines
// may belong to different outer indices); offsets are 32-bit (the launcher
// rejects operands of 2^31 entries or more), which keeps a unit's indices in
// one register each until the write-back.
template <typename C, typename T, bool UPDATE>
struct ColSource {
  static constexpr bool kWriteBack = UPDATE;
  const C* __restrict__ in;
  const C* __restrict__ pold;
  C* __restrict__ pnew;
  const int* off;
  T beta;
  int inner;        // row stride
  int half, M, width;
  __device__ __forceinline__ int index(int t, int n, bool& ok) const {
    const int r = n <= half ? n : (n >= M - half ? n - M : M);   // row offset from the centre
    ok = r != M && t < width;
    return off[t] + (r + half) * inner;
  }
  __device__ __forceinline__ C operator()(int t, int n) const {
    bool ok;
    const int idx = index(t, n, ok);
    C v = mk(T(0), T(0));
    if (ok) {
      v = in[idx];
      if constexpr (UPDATE) {
        const C po = pold[idx];
        v = mk(v.x + beta * po.x, v.y + beta * po.y);
      }
    }
    return v;
  }
  __device__ __forceinline__ void write_back(int t, int n, C v) const {
    bool ok;
    const int idx = index(t, n, ok);
    if (ok) pnew[idx] = v;
  }
};

template <typename T, int TW, int SIGN, int MODE, int MCT = 0>
__device__ __forceinline__ void col_body(const ColArgs& a, const FftPlan& pl, int64_t bid) {
  using C = typename CT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  __shared__ PassSmem st;
  if (a.st != nullptr && a.st->done != RUNNING) return;
  const int npass = load_passes<C>(st, pl);

  const int M = MCT != 0 ? MCT : pl.M;
  // runtime plans: tile (o, j0 .. j0 + TW) of one outer index; size-specialised
  // transforms: TW consecutive columns of the flattened (outer, inner) range,
  // so that no CTA is spent on the ragged end of each outer index
  const int64_t tiles = (a.inner + TW - 1) / TW;
  const int64_t o = MCT != 0 ? 0 : bid / tiles;
  const int64_t j0 = MCT != 0 ? 0 : (bid % tiles) * TW;
  int width = static_cast<int>(a.inner - j0 < TW ? a.inner - j0 : TW);
  __shared__ int s_in[MCT != 0 ? TW : 1], s_out[MCT != 0 ? TW : 1];
  if constexpr (MCT != 0) {
    const int64_t ncols = a.outer * a.inner;
    const int64_t g0 = bid * TW;
    width = static_cast<int>(ncols - g0 < TW ? ncols - g0 : TW);
    const int64_t rows_in = SIGN > 0 ? a.Lin : M;
    const int64_t rows_out = SIGN > 0 ? M : a.Lout;
    if (threadIdx.x < TW) {
      const int64_t g = g0 + (static_cast<int>(threadIdx.x) < width ? threadIdx.x : width - 1);
      const int64_t oo = g / a.inner, jj = g - oo * a.inner;
      s_in[threadIdx.x] = static_cast<int>(oo * rows_in * a.inner + jj);
      s_out[threadIdx.x] = static_cast<int>(oo * rows_out * a.inner + jj);
    }
    __syncthreads();
  }
  const C* __restrict__ tw = twtab<C>(pl);
  const int* __restrict__ perm = MCT != 0 ? pl.perm_ct : pl.perm;

  if constexpr (MCT != 0 && SIGN > 0) {
    // The size-specialised transform reads its input rows straight from global
    // memory in its first pass (input n of line t is row i(n) of the tile,
    // zero outside the padded range; p = r + beta p_old is formed and written
    // back on the way).
    const C* __restrict__ in = static_cast<const C*>(a.in);
    const int Lin = a.Lin;
    const int half = (Lin - 1) / 2;
    T beta = T(0);
    if constexpr (MODE == COL_PUPDATE) beta = static_cast<T>(a.st->beta);
    const C* pold = nullptr;
    C* pnew = nullptr;
    if constexpr (MODE == COL_PUPDATE) {
      pold = static_cast<const C*>(a.pold);
      pnew = static_cast<C*>(a.pnew);
    }
    ColSource<C, T, MODE == COL_PUPDATE> src{in, pold, pnew, s_in, beta, static_cast<int>(a.inner), half, M, width};
    fft_dit_ct_src<+1, TW, col_threads<T, TW, MCT, MODE>(), MCT>(buf, tw, src);
    C* __restrict__ out = static_cast<C*>(a.out);
    for (int u = threadIdx.x; u < M * TW; u += blockDim.x) {
      const int t = u % TW;
      const int m = u / TW;
      if (t < width) out[s_out[t] + m * static_cast<int>(a.inner)] = buf[m * TW + t];
    }
  } else if constexpr (MCT != 0) {
    // forward, size-specialised: natural-order input copied in, the last
    // pass hands the kept frequencies (scaled by 1/M) straight to global memory
    const C* __restrict__ in = static_cast<const C*>(a.in);
    for (int u = threadIdx.x; u < M * TW; u += blockDim.x) {
      const int t = u % TW;
      const int m = u / TW;
      if (t < width) cp_async<sizeof(C)>(buf + u, in + (s_in[t] + m * static_cast<int>(a.inner)));
      else buf[u] = mk(T(0), T(0));
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    C* __restrict__ out = static_cast<C*>(a.out);
    const int Lout = a.Lout;
    const int half = (Lout - 1) / 2;
    const T inv = T(1) / T(M);
    auto snk = [&](int t, int n, C v) {
      const int i = n <= half ? n + half : (n >= M - half ? n - M + half : -1);
      if (i >= 0 && t < width) out[s_out[t] + i * static_cast<int>(a.inner)] = inv * v;
    };
    fft_dif_ct_snk<-1, TW, col_threads<T, TW, MCT, MODE>(), MCT>(buf, tw, snk);
  } else if (SIGN > 0) {
    const C* __restrict__ in = static_cast<const C*>(a.in);
    const int Lin = a.Lin;
    const int half = (Lin - 1) / 2;
    // zero the frequencies the input does not reach: k = half+1 .. M-half-1
    for (int u = threadIdx.x; u < (M - Lin) * TW; u += blockDim.x) {
      const int t = u % TW;
      const int k = half + 1 + u / TW;
      buf[bix<MCT, C>(__ldg(&perm[k]) * TW + t)] = mk(T(0), T(0));
    }
    if (MODE == COL_PLAIN) {
      for (int u = threadIdx.x; u < Lin * TW; u += blockDim.x) {
        const int t = u % TW;
        const int i = u / TW;
        int k = i - half;
        if (k < 0) k += M;
        C* dst = buf + bix<MCT, C>(__ldg(&perm[k]) * TW + t);
        if (t < width) cp_async<sizeof(C)>(dst, in + (o * Lin + i) * a.inner + j0 + t);
        else *dst = mk(T(0), T(0));
      }
      cp_async_commit();
      cp_async_wait<0>();
    } else {
      // p = r + beta p_old, written back and scattered; K entries per thread
      // are loaded before any is used so that their latencies overlap
      constexpr int K = 4;
      const T beta = static_cast<T>(a.st->beta);
      const C* __restrict__ pold = static_cast<const C*>(a.pold);
      C* pnew = static_cast<C*>(a.pnew);
      for (int u0 = threadIdx.x; u0 < Lin * TW; u0 += K * blockDim.x) {
        C v[K], po[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int u = u0 + q * blockDim.x;
          const int t = u % TW;
          const int i = u / TW;
          v[q] = mk(T(0), T(0));
          po[q] = mk(T(0), T(0));
          if (u < Lin * TW && t < width) {
            const int64_t idx = (o * Lin + i) * a.inner + j0 + t;
            v[q] = in[idx];
            po[q] = pold[idx];
          }
        }
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int u = u0 + q * blockDim.x;
          if (u < Lin * TW) {
            const int t = u % TW;
            const int i = u / TW;
            const C w = mk(v[q].x + beta * po[q].x, v[q].y + beta * po[q].y);
            if (t < width) pnew[(o * Lin + i) * a.inner + j0 + t] = w;
            int k = i - half;
            if (k < 0) k += M;
            buf[bix<MCT, C>(__ldg(&perm[k]) * TW + t)] = (t < width) ? w : mk(T(0), T(0));
          }
        }
      }
    }
    __syncthreads();
    fft_dit<+1, TW>(buf, st, npass, M, tw);
    C* __restrict__ out = static_cast<C*>(a.out);
    for (int u = threadIdx.x; u < M * TW; u += blockDim.x) {
      const int t = u % TW;
      const int m = u / TW;
      if (t < width) out[(o * M + m) * a.inner + j0 + t] = buf[bix<MCT, C>(m * TW + t)];
    }
  } else {
    const C* __restrict__ in = static_cast<const C*>(a.in);
    for (int u = threadIdx.x; u < M * TW; u += blockDim.x) {
      const int t = u % TW;
      const int m = u / TW;
      if (t < width) cp_async<sizeof(C)>(buf + bix<MCT, C>(u), in + (o * M + m) * a.inner + j0 + t);
      else buf[bix<MCT, C>(u)] = mk(T(0), T(0));
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    fft_dif<-1, TW>(buf, st, npass, M, tw);
    C* __restrict__ out = static_cast<C*>(a.out);
    const int Lout = a.Lout;
    const int half = (Lout - 1) / 2;
    const T inv = T(1) / T(M);
    for (int u = threadIdx.x; u < Lout * TW; u += blockDim.x) {
      const int t = u % TW;
      const int i = u / TW;
      if (t < width) {
        int k = i - half;
        if (k < 0) k += M;
        C v = buf[bix<MCT, C>(__ldg(&perm[k]) * TW + t)];
        out[(o * Lout + i) * a.inner + j0 + t] = inv * v;
      }
    }
  }
}


constexpr int kColThreads32 = 512;
constexpr int kColThreads64 = 256;

template <typename T, int TW, int SIGN, int MODE, int MCT = 0>
__global__ void __launch_bounds__(col_threads<T, TW, MCT, MODE>(), col_min_blocks<T, TW, MCT, MODE>())
    col_kernel(ColArgs a, FftPlan pl) {
  col_body<T, TW, SIGN, MODE, MCT>(a, pl, blockIdx.x);
}

// Index of the work item owning block `b` (items sorted by block_begin).
template <typename Item>
__device__ __forceinline__ int find_item(const Item* items, int n, int64_t b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].block_begin <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Many operands (instances, solves) in one launch: each item owns a
// contiguous range of blocks.
template <typename T, int TW, int SIGN, int MODE>
__global__ void __launch_bounds__(sizeof(T) == 8 ? kColThreads64 : kColThreads32)
    col_kernel_batch(const ColItem* __restrict__ items, int n) {
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = find_item(items, n, blockIdx.x);
  __syncthreads();
  const ColItem& it = items[s_item];
  col_body<T, TW, SIGN, MODE>(it.a, *it.pl, blockIdx.x - it.block_begin);
}

template <typename T, int TW, int SIGN, int MODE, int MCT = 0>
inline ghb_status launch_col_t(const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  using C = typename CT<T>::type;
  const size_t smem = col_smem_bytes(pl.M, TW, sizeof(C));
  static std::atomic<unsigned long long> attr_mask{0};
  TRY_STATUS(ensure_dyn_smem(col_kernel<T, TW, SIGN, MODE, MCT>, 220 * 1024, attr_mask));
  const int64_t tiles = (a.inner + TW - 1) / TW;
  const int64_t grid = MCT != 0 ? (a.outer * a.inner + TW - 1) / TW : tiles * a.outer;
  if (MCT != 0 && a.outer * std::max<int64_t>(std::max<int64_t>(a.Lin, a.Lout), pl.M) * a.inner >= (int64_t(1) << 31)) {
    set_error("column pass operand of 2^31 entries or more");
    return GHB_ERR_INVALID;
  }
  const int threads = MCT != 0 ? col_threads<T, TW, MCT, MODE>()
                               : ((sizeof(T) == 4 && pl.M * TW >= 2048) ? kColThreads32 : 256);
  col_kernel<T, TW, SIGN, MODE, MCT><<<static_cast<unsigned>(grid), threads, smem, s>>>(a, pl);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

// All sign/mode variants of one precision and tile width.
template <typename T, int TW, int MCT = 0>
ghb_status launch_col_tw(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  if (sign > 0)
    return mode == COL_PUPDATE ? launch_col_t<T, TW, +1, COL_PUPDATE, MCT>(a, pl, s)
                               : launch_col_t<T, TW, +1, COL_PLAIN, MCT>(a, pl, s);
  return launch_col_t<T, TW, -1, COL_PLAIN, MCT>(a, pl, s);
}

template <typename T, int TW, int SIGN, int MODE>
inline ghb_status launch_col_batch_t(const ColItem* items, int n, int64_t blocks, size_t smem, int threads,
                                     cudaStream_t s) {
  static std::atomic<unsigned long long> attr_mask{0};
  TRY_STATUS(ensure_dyn_smem(col_kernel_batch<T, TW, SIGN, MODE>, 220 * 1024, attr_mask));
  // threads <= 0: the kernel's full block; fewer for short transforms, whose
  // passes have fewer butterflies than a full block has threads
  const int full = sizeof(T) == 4 ? kColThreads32 : kColThreads64;
  const int nt = (threads > 0 && threads < full) ? threads : full;
  col_kernel_batch<T, TW, SIGN, MODE><<<static_cast<unsigned>(blocks), nt, smem, s>>>(items, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

template <typename T, int TW>
ghb_status launch_col_batch_tw(int sign, int mode, const ColItem* items, int n, int64_t blocks, size_t smem, int threads,
                               cudaStream_t s) {
  if (sign > 0)
    return mode == COL_PUPDATE ? launch_col_batch_t<T, TW, +1, COL_PUPDATE>(items, n, blocks, smem, threads, s)
                               : launch_col_batch_t<T, TW, +1, COL_PLAIN>(items, n, blocks, smem, threads, s);
  return launch_col_batch_t<T, TW, -1, COL_PLAIN>(items, n, blocks, smem, threads, s);
}

// ---------------------------------------------------------------------------
// row pass
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// row pass
// ---------------------------------------------------------------------------
struct LineDesc {
  int64_t row;
  int field;
  int comp;
  int valid;
};

// Field f of a row pass.  Selects rather than an index into the argument's
// array: a run-time index into a kernel parameter makes the compiler copy the
// whole argument to local memory and load the pointer from there (the FP32
// last-axis pass at M = 4374: 164 -> 145 us without that copy and without
// the per-entry line masks of its staged spectra).
__device__ __forceinline__ void* row_field(const RowArgs& a, int f) {
  return f == 0 ? a.t[0] : (f == 1 ? a.t[1] : a.t[2]);
}

template <typename T, int NL, int MODE>
__device__ __forceinline__ void row_body(const RowArgs& a, const FftPlan& pl, int rows_per_cta,
                                         int64_t bid, int64_t nb) {
  using C = typename CT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  __shared__ PassSmem st;
  __shared__ LineDesc ld[2 * NL];
  __shared__ double red[32];
  __shared__ bool last;
  if (a.st != nullptr && a.st->done != RUNNING) return;
  const int npass = load_passes<C>(st, pl);

  const int M = pl.M;
  const int H = a.H;
  const int per_row = a.nfields * a.ncomp;
  const int nrl = rows_per_cta * per_row;   // real lines per row group
  const int64_t groups = (a.rows + rows_per_cta - 1) / rows_per_cta;
  const C* __restrict__ tw = twtab<C>(pl);
  const int* __restrict__ perm = pl.perm;
  double g[6] = {0, 0, 0, 0, 0, 0};       // ENERGY: upper triangle of F x F, F <= 3

  for (int64_t grp = bid; grp < groups; grp += nb) {
    const int64_t row0 = grp * rows_per_cta;
    if (threadIdx.x < 2 * NL) {
      const int rho = threadIdx.x;
      LineDesc d;
      d.row = row0 + rho / per_row;
      d.field = (rho / a.ncomp) % a.nfields;
      d.comp = rho % a.ncomp;
      d.valid = (rho < nrl) && (d.row < a.rows);
      ld[rho] = d;
    }
    for (int u = threadIdx.x; u < static_cast<int>(padded_elems<C>(M * NL)); u += blockDim.x) buf[u] = mk(T(0), T(0));
    __syncthreads();

    // Hermitian completion of each pair of half spectra: Z(k) = X0(k) + i X1(k),
    // Z(-k) = conj X0(k) + i conj X1(k); scattered to digit-reversed positions.
    for (int u = threadIdx.x; u < NL * H; u += blockDim.x) {
      const int j = (NL == 1) ? 0 : u % NL;
      const int k = (NL == 1) ? u : u / NL;
      const LineDesc d0 = ld[2 * j], d1 = ld[2 * j + 1];
      C A = mk(T(0), T(0)), B = mk(T(0), T(0));
      if (d0.valid)
        A = static_cast<const C*>(row_field(a, d0.field))[d0.comp * a.comp_stride + d0.row * H + k];
      if (d1.valid)
        B = static_cast<const C*>(row_field(a, d1.field))[d1.comp * a.comp_stride + d1.row * H + k];
      buf[pidx<C>(__ldg(&perm[k]) * NL + j)] = mk(A.x - B.y, A.y + B.x);
      if (k > 0) buf[pidx<C>(__ldg(&perm[M - k]) * NL + j)] = mk(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    fft_dit<+1, NL>(buf, st, npass, M, tw);

    if (MODE == ROW_MATVEC) {
      const T* __restrict__ am = static_cast<const T*>(a.a);
      for (int u = threadIdx.x; u < NL * M; u += blockDim.x) {
        const int j = (NL == 1) ? 0 : u % NL;
        const int m = (NL == 1) ? u : u / NL;
        const LineDesc d0 = ld[2 * j], d1 = ld[2 * j + 1];
        C z = buf[pidx<C>(m * NL + j)];
        const T a0 = d0.valid ? am[d0.row * M + m] : T(0);
        const T a1 = d1.valid ? am[d1.row * M + m] : T(0);
        buf[pidx<C>(m * NL + j)] = mk(a0 * z.x, a1 * z.y);
      }
      __syncthreads();
      fft_dif<-1, NL>(buf, st, npass, M, tw);
      const T sc = T(0.5) / T(M);
      for (int u = threadIdx.x; u < NL * H; u += blockDim.x) {
        const int j = (NL == 1) ? 0 : u % NL;
        const int k = (NL == 1) ? u : u / NL;
        const LineDesc d0 = ld[2 * j], d1 = ld[2 * j + 1];
        const C W = buf[pidx<C>(__ldg(&perm[k]) * NL + j)];
        const C Wm = buf[pidx<C>(__ldg(&perm[k == 0 ? 0 : M - k]) * NL + j)];
        if (d0.valid)
          static_cast<C*>(row_field(a, d0.field))[d0.comp * a.comp_stride + d0.row * H + k] =
              mk(sc * (W.x + Wm.x), sc * (W.y - Wm.y));
        if (d1.valid)
          static_cast<C*>(row_field(a, d1.field))[d1.comp * a.comp_stride + d1.row * H + k] =
              mk(sc * (W.y + Wm.y), sc * (Wm.x - W.x));
      }
    } else if (MODE == ROW_TOREAL) {
      T* __restrict__ out = static_cast<T*>(a.out_real);
      for (int u = threadIdx.x; u < NL * M; u += blockDim.x) {
        const int j = (NL == 1) ? 0 : u % NL;
        const int m = (NL == 1) ? u : u / NL;
        const LineDesc d0 = ld[2 * j], d1 = ld[2 * j + 1];
        const C z = buf[pidx<C>(m * NL + j)];
        if (d0.valid) out[d0.row * M + m] = z.x;
        if (d1.valid) out[d1.row * M + m] = z.y;
      }
    } else {  // ROW_ENERGY: one row per group, lines ordered (field, comp)
      const T* __restrict__ am = static_cast<const T*>(a.a);
      const int F = a.nfields, NC = a.ncomp;
      const bool ok = ld[0].valid;
      for (int m = threadIdx.x; ok && m < M; m += blockDim.x) {
        const double am_ = static_cast<double>(am[ld[0].row * M + m]);
        double u[10];
#pragma unroll
        for (int r = 0; r < 2 * NL; ++r) {
          const C z = buf[pidx<C>(m * NL + (r >> 1))];
          u[r] = static_cast<double>((r & 1) ? z.y : z.x);
        }
        int e = 0;
        for (int f = 0; f < F; ++f)
          for (int h2 = f; h2 < F; ++h2, ++e) {
            double s = 0.0;
            for (int c = 0; c < NC; ++c) s += u[f * NC + c] * u[h2 * NC + c];
            g[e] += am_ * s;
          }
      }
    }
    __syncthreads();
  }

  if (MODE == ROW_ENERGY) {
    const int F = a.nfields;
    const int ne = F * (F + 1) / 2;
    for (int e = 0; e < ne; ++e) {
      const double v = block_sum(g[e], red);
      if (threadIdx.x == 0) a.partials[bid * 6 + e] = v;
    }
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned int t = atomicAdd(a.ticket, 1u);
      last = (t == nb - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      for (int e = 0; e < ne; ++e) {
        double v = 0.0;
        for (int64_t b = threadIdx.x; b < nb; b += blockDim.x)
          v += __ldcg(&a.partials[b * 6 + e]);
        v = block_sum(v, red);
        if (threadIdx.x == 0) {
          int ee = 0;
          for (int f = 0; f < F; ++f)
            for (int h2 = f; h2 < F; ++h2, ++ee)
              if (ee == e) {
                a.gram[f * F + h2] = v * a.scale;
                a.gram[h2 * F + f] = v * a.scale;
              }
        }
      }
      if (threadIdx.x == 0) *a.ticket = 0u;
    }
  }
}

constexpr int kRowThreads = 256;

// The size-specialised FP32 last-axis kernels read A_M from global memory in
// their fused pass (coalesced: a warp's threads hold consecutive entries)
// instead of staging it, which frees shared memory for a fourth CTA per SM,
// and run 192 threads per CTA (a radix-27 pass at M = 4374 has 162
// butterflies per line).  At M = 4374: 173 us per launch against 184 us with
// the staged A_M and 256 threads; at M = 270 (15 lines per CTA): 300 us
// against 334 us.
template <typename T, int MCT>
__host__ __device__ constexpr bool row_streams_multiplier() {
  return MCT != 0 && sizeof(T) == 4;
}
template <typename T, int MCT>
__host__ __device__ constexpr int row_threads() {
  return row_streams_multiplier<T, MCT>() ? 192 : kRowThreads;
}

// FP32: at most 85 registers so that three CTAs share an SM (measured 19 %
// faster at M = 4374 than two CTAs of 128 registers).
// Operator pass with staged inputs (MATVEC only; used when the staging fits
// in shared memory).  The CTA loops over row groups; the next group's half
// spectra are copied asynchronously into a staging area while the current
// group is transformed, and the next group's multiplier row while the current
// one is transformed back:
//
//   smem = [ transform buffer | staged half spectra [2 NL][H] | staged A_M rows [rows][M] ]
//
// Copy groups in flight per thread: at the multiply, {A_M(g), spectra(g+1)};
// wait_group 1 therefore waits for A_M(g) alone.  Kernels that stream A_M
// (row_streams_multiplier) have no A_M area and commit empty A_M groups, so the
// count is the same.
// Staged half spectra: the two real lines of complex line j side by side,
// entry (j, k) at pair index j * row_pair_stride(H) + k (an odd stride, so that
// threads of consecutive lines reading the same k fall on different banks).
__host__ __device__ inline int row_pair_stride(int H) { return H | 1; }
template <typename T>
__host__ __device__ inline size_t row_buf_elems(int M, int NL) {   // rounded to 16 bytes
  using C = typename CT<T>::type;
  const size_t e = padded_elems<C>(static_cast<size_t>(M) * NL);
  return sizeof(C) >= 16 ? e : (e + 1) & ~static_cast<size_t>(1);
}
template <typename T, int NL>
__host__ __device__ inline size_t row_staged_smem(int M, int H, int rows_per_cta) {
  using C = typename CT<T>::type;
  return row_buf_elems<T>(M, NL) * sizeof(C) + static_cast<size_t>(2 * NL) * row_pair_stride(H) * sizeof(C) +
         static_cast<size_t>(rows_per_cta) * M * sizeof(T);
}

// Input of the size-specialised last-axis transforms: entry n of complex line
// j is the Hermitian completion of the two staged half spectra X0, X1 of its
// real lines (X(k), k = 0 .. H-1; line pairs at stride SH):
//     Z(n) = X0(n) + i X1(n)                      n < H,
//     Z(n) = conj X0(M-n) + i conj X1(M-n)        n > M - H,
//     0                                           otherwise.
// With RANGED, ranged() decides for a whole range of n at once (see
// ct_ranged): in the first pass at M = 4374, N = 2187 every range but two lies
// entirely below H, entirely above M - H or entirely in the zeros.  Measured
// per kernel: FP64 last-axis pass 4310 -> 4256 us at M = 4374 and 4204 -> 4125
// us at M = 270, FP32 209 -> 204 us at M = 270, but FP32 144 -> 148 us at
// M = 4374, which therefore keeps the test per entry.
template <typename C, typename Pair, bool RANGED>
struct RowSource {
  static constexpr bool kRanged = RANGED;
  const Pair* spair;
  int SH, H, M;
  __device__ __forceinline__ C lo(int j, int k) const {
    const Pair v = spair[j * SH + k];   // both real lines in one load
    return mk(v.a.x - v.b.y, v.a.y + v.b.x);
  }
  __device__ __forceinline__ C hi(int j, int k) const {
    const Pair v = spair[j * SH + k];
    return mk(v.a.x + v.b.y, v.b.x - v.a.y);
  }
  __device__ __forceinline__ C operator()(int j, int n) const {
    using T = decltype(C{}.x);
    const bool l = n < H, h = n > M - H;
    const int k = l ? n : M - n;
    C A = mk(T(0), T(0)), B = mk(T(0), T(0));
    if (l || h) {
      const Pair v = spair[j * SH + k];
      A = v.a;
      B = v.b;
    }
    return l ? mk(A.x - B.y, A.y + B.x) : mk(A.x + B.y, B.x - A.y);
  }
  __device__ __forceinline__ C ranged(int j, int nb, int n0, int span) const {
    using T = decltype(C{}.x);
    if (n0 + span - 1 < H) return lo(j, nb + n0);
    if (n0 > M - H) return hi(j, M - n0 - nb);
    if (n0 >= H && n0 + span - 1 <= M - H) return mk(T(0), T(0));
    return (*this)(j, nb + n0);
  }
};

template <typename T, int NL, int MCT = 0>
__device__ __forceinline__ void row_matvec_staged(const RowArgs& a, const FftPlan& pl, int rows_per_cta,
                                                  int64_t bid, int64_t nb) {
  using C = typename CT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassSmem st;
  __shared__ LineDesc ld[2 * NL], ldn[2 * NL];   // this group's lines, the next group's
  // per complex line j of this group: bit 0 / bit 1 = real line 2j / 2j+1 is
  // valid; offsets of their A_M rows (in `am`, or in the staged rows `sa`)
  __shared__ int lmask[NL];
  __shared__ int2 lrow[NL];
  if (a.st != nullptr && a.st->done != RUNNING) return;
  const int npass = load_passes<C>(st, pl);

  const int M = MCT != 0 ? MCT : pl.M;
  const int H = a.H;
  const int per_row = a.nfields * a.ncomp;
  const int nrl = rows_per_cta * per_row;
  const int64_t groups = (a.rows + rows_per_cta - 1) / rows_per_cta;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* sin = buf + row_buf_elems<T>(M, NL);
  const int SH = row_pair_stride(H);
  T* sa = reinterpret_cast<T*>(sin + 2 * NL * SH);
  struct alignas(sizeof(C) >= 16 ? 16 : 2 * sizeof(C)) Pair {
    C a, b;
  };
  const Pair* spair = reinterpret_cast<const Pair*>(sin);
  const C* __restrict__ tw = twtab<C>(pl);
  const int* __restrict__ perm = MCT != 0 ? pl.perm_ct : pl.perm;
  const T* __restrict__ am = static_cast<const T*>(a.a);

  auto desc = [&](int64_t grp, int rho) {
    LineDesc d;
    d.row = grp * rows_per_cta + rho / per_row;
    d.field = (rho / a.ncomp) % a.nfields;
    d.comp = rho % a.ncomp;
    d.valid = (rho < nrl) && (d.row < a.rows);
    return d;
  };
  // Copies of the half spectra of the lines described by L[0 .. 2NL) into the
  // staging area; a line that is not valid (past the last row) gets zeros,
  // so that the transforms read the staged pairs without masks.  Long rows
  // (H >= the block): line by line, the block striding over k.  Short rows:
  // one flat loop over (line, k), the line and k of a thread advanced by the
  // block size each step (no division per entry).
  auto issue_from = [&](const LineDesc* L) {
    if (H >= static_cast<int>(blockDim.x)) {
#pragma unroll 1
      for (int rho = 0; rho < 2 * NL; ++rho) {
        const LineDesc d = L[rho];
        C* dst = sin + (rho >> 1) * 2 * SH + (rho & 1);
        if (!d.valid) {
          for (int k = threadIdx.x; k < H; k += blockDim.x) dst[2 * k] = mk(T(0), T(0));
          continue;
        }
        const C* src = static_cast<const C*>(row_field(a, d.field)) + d.comp * a.comp_stride + d.row * H;
        for (int k = threadIdx.x; k < H; k += blockDim.x) cp_async<sizeof(C)>(dst + 2 * k, src + k);
      }
      return;
    }
    const int step_r = static_cast<int>(blockDim.x) / H, step_k = static_cast<int>(blockDim.x) - step_r * H;
    int rho = static_cast<int>(threadIdx.x) / H;
    int k = static_cast<int>(threadIdx.x) - rho * H;
    while (rho < 2 * NL) {
      const LineDesc d = L[rho];
      C* dst = sin + ((rho >> 1) * SH + k) * 2 + (rho & 1);
      if (d.valid)
        cp_async<sizeof(C)>(dst, static_cast<const C*>(row_field(a, d.field)) + d.comp * a.comp_stride + d.row * H + k);
      else
        *dst = mk(T(0), T(0));
      rho += step_r;
      k += step_k;
      if (k >= H) {
        k -= H;
        ++rho;
      }
    }
  };
  auto issue_multiplier = [&](int64_t grp) {
    if constexpr (!row_streams_multiplier<T, MCT>()) {   // else read in the fused pass instead
      for (int r = 0; r < rows_per_cta; ++r) {
        const int64_t row = grp * rows_per_cta + r;
        if (row >= a.rows) break;
        for (int m = threadIdx.x; m < M; m += blockDim.x) cp_async<sizeof(T)>(sa + r * M + m, am + row * M + m);
      }
    }
  };

  int64_t grp = bid;
  if (grp < groups) {
    if (threadIdx.x < 2 * NL) ldn[threadIdx.x] = desc(grp, threadIdx.x);
    __syncthreads();
    issue_from(ldn);
    cp_async_commit();
    issue_multiplier(grp);
    cp_async_commit();
    __syncthreads();   // ldn is rewritten at the top of the loop
  }
  for (; grp < groups; grp += nb) {
    // every thread has issued the copies of ldn's lines (barriers since then)
    if (threadIdx.x < 2 * NL) {
      ld[threadIdx.x] = desc(grp, threadIdx.x);
      ldn[threadIdx.x] = desc(grp + nb, threadIdx.x);
    }
    if (threadIdx.x < NL) {
      const int j = threadIdx.x;
      const LineDesc d0 = desc(grp, 2 * j), d1 = desc(grp, 2 * j + 1);
      lmask[j] = (d0.valid ? 1 : 0) | (d1.valid ? 2 : 0);
      if constexpr (row_streams_multiplier<T, MCT>())
        lrow[j] = make_int2(d0.valid ? static_cast<int>(d0.row * M) : 0, d1.valid ? static_cast<int>(d1.row * M) : 0);
      else
        lrow[j] = make_int2(((2 * j) / per_row) * M, ((2 * j + 1) / per_row) * M);
    }
    cp_async_wait<1>();          // spectra(g) are in; A_M(g) may still be in flight
    __syncthreads();

    // Hermitian completion of each pair of half spectra (Z(k) = X0(k) + i X1(k),
    // Z(-k) = conj X0(k) + i conj X1(k)) into digit-reversed positions, and
    // zeros at the frequencies the spectra do not reach (k = H .. M-H).  The
    // size-specialised transform reads the completed spectrum directly in its
    // first pass instead.
    if constexpr (MCT != 0) {
      // the staged pairs hold zeros for a line that is not valid
      constexpr bool ranged = sizeof(T) == 8 || MCT == 72 || MCT == 135 || MCT == 270;
      const RowSource<C, Pair, ranged> src{spair, SH, H, M};
      // multiply by A_M between the transforms, in registers
      auto mul = [&](int j, int m, C z) -> C {
        T a0 = T(0), a1 = T(0);
        const int2 ro = lrow[j];
        if constexpr (row_streams_multiplier<T, MCT>()) {
          // a line that is not valid reads row 0 (in bounds, finite) and is
          // not stored; its zero input keeps the other line of the pair exact
          a0 = __ldg(&am[ro.x + m]);
          a1 = __ldg(&am[ro.y + m]);
        } else {
          const int msk = lmask[j];
          if (msk & 1) a0 = sa[ro.x + m];
          if (msk & 2) a1 = sa[ro.y + m];
        }
        return mk(a0 * z.x, a1 * z.y);
      };
      auto after_first = [&]() {   // the staged spectra are read: stage the next group's
        if (grp + nb < groups) issue_from(ldn);
        cp_async_commit();
      };
      auto before_fused = [&]() {  // A_M(g) is in; spectra(g+1) may still be in flight
        cp_async_wait<1>();
        __syncthreads();
      };
      auto after_fused = [&]() {   // the staged A_M is read: stage the next group's
        if (grp + nb < groups) issue_multiplier(grp + nb);
        cp_async_commit();
      };
      ct_inverse_scale_forward<+1, -1, NL, row_threads<T, MCT>(), MCT>(buf, tw, src, mul, after_first, before_fused,
                                                             after_fused);   // ends with a barrier
    } else {
    for (int u = threadIdx.x; u < NL * H; u += blockDim.x) {
      const int j = (NL == 1) ? 0 : u % NL;
      const int k = (NL == 1) ? u : u / NL;
      const Pair v = spair[j * SH + k];
      const int msk = lmask[j];
      const C A = (msk & 1) ? v.a : mk(T(0), T(0));
      const C B = (msk & 2) ? v.b : mk(T(0), T(0));
      buf[bix<MCT, C>(__ldg(&perm[k]) * NL + j)] = mk(A.x - B.y, A.y + B.x);
      if (k > 0) buf[bix<MCT, C>(__ldg(&perm[M - k]) * NL + j)] = mk(A.x + B.y, B.x - A.y);
    }
    for (int u = threadIdx.x; u < NL * (M - 2 * H + 1); u += blockDim.x) {
      const int j = (NL == 1) ? 0 : u % NL;
      const int k = H + ((NL == 1) ? u : u / NL);
      buf[bix<MCT, C>(__ldg(&perm[k]) * NL + j)] = mk(T(0), T(0));
    }
    __syncthreads();
    if (grp + nb < groups) issue_from(ldn);   // staging is free again
    fft_dit<+1, NL>(buf, st, npass, M, tw);
    cp_async_commit();

    cp_async_wait<1>();          // A_M(g) is in; spectra(g+1) may still be in flight
    __syncthreads();
    for (int u = threadIdx.x; u < NL * M; u += blockDim.x) {
      const int j = (NL == 1) ? 0 : u % NL;
      const int m = (NL == 1) ? u : u / NL;
      const int msk = lmask[j];
      const int2 ro = lrow[j];
      const C z = buf[bix<MCT, C>(m * NL + j)];
      const T a0 = (msk & 1) ? sa[ro.x + m] : T(0);
      const T a1 = (msk & 2) ? sa[ro.y + m] : T(0);
      buf[bix<MCT, C>(m * NL + j)] = mk(a0 * z.x, a1 * z.y);
    }
    __syncthreads();
    if (grp + nb < groups) issue_multiplier(grp + nb);
    cp_async_commit();
    fft_dif<-1, NL>(buf, st, npass, M, tw);
    }
    const T sc = T(0.5) / T(M);
    for (int u = threadIdx.x; u < NL * H; u += blockDim.x) {
      const int j = (NL == 1) ? 0 : u % NL;
      const int k = (NL == 1) ? u : u / NL;
      const LineDesc d0 = ld[2 * j], d1 = ld[2 * j + 1];
      const C W = buf[bix<MCT, C>(__ldg(&perm[k]) * NL + j)];
      const C Wm = buf[bix<MCT, C>(__ldg(&perm[k == 0 ? 0 : M - k]) * NL + j)];
      if (d0.valid)
        static_cast<C*>(row_field(a, d0.field))[d0.comp * a.comp_stride + d0.row * H + k] =
            mk(sc * (W.x + Wm.x), sc * (W.y - Wm.y));
      if (d1.valid)
        static_cast<C*>(row_field(a, d1.field))[d1.comp * a.comp_stride + d1.row * H + k] =
            mk(sc * (W.y + Wm.y), sc * (Wm.x - W.x));
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <typename T, int NL, int MCT = 0>
__global__ void __launch_bounds__(row_threads<T, MCT>(), sizeof(T) == 4 ? (row_streams_multiplier<T, MCT>() ? 4 : 3) : 1)
    row_kernel_staged(RowArgs a, FftPlan pl, int rows_per_cta) {
  row_matvec_staged<T, NL, MCT>(a, pl, rows_per_cta, blockIdx.x, gridDim.x);
}

template <typename T, int NL, int MODE>
__global__ void __launch_bounds__(kRowThreads, sizeof(T) == 4 ? 3 : 1)
    row_kernel(RowArgs a, FftPlan pl, int rows_per_cta) {
  row_body<T, NL, MODE>(a, pl, rows_per_cta, blockIdx.x, gridDim.x);
}

template <typename T, int NL, int MODE>
__global__ void __launch_bounds__(kRowThreads, sizeof(T) == 4 ? 3 : 1)
    row_kernel_batch(const RowItem* __restrict__ items, int n) {
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = find_item(items, n, blockIdx.x);
  __syncthreads();
  const RowItem& it = items[s_item];
  row_body<T, NL, MODE>(it.a, *it.pl, it.rows_per_cta, blockIdx.x - it.block_begin, it.nblocks);
}

template <typename T, int NL, int MODE>
inline ghb_status launch_row_batch_t(const RowItem* items, int n, int64_t blocks, size_t smem, int threads,
                                     cudaStream_t s) {
  static std::atomic<unsigned long long> attr_mask{0};
  TRY_STATUS(ensure_dyn_smem(row_kernel_batch<T, NL, MODE>, 200 * 1024, attr_mask));
  const int nt = (MODE == ROW_MATVEC && threads > 0 && threads < kRowThreads) ? threads : kRowThreads;
  row_kernel_batch<T, NL, MODE><<<static_cast<unsigned>(blocks), nt, smem, s>>>(items, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

template <typename T, int NL, int MODE, int MCT = 0>
inline ghb_status launch_row_t(const RowArgs& a, const FftPlan& pl, int rows_per_cta,
                               cudaStream_t s) {
  using C = typename CT<T>::type;
  const size_t smem = padded_elems<C>(static_cast<size_t>(pl.M) * NL) * sizeof(C);
  static std::atomic<unsigned long long> attr_mask{0};
  TRY_STATUS(ensure_dyn_smem(row_kernel<T, NL, MODE>, 200 * 1024, attr_mask));
  if (smem > 200 * 1024) {
    set_error("row transform too large for one CTA: M=" + std::to_string(pl.M));
    return GHB_ERR_INVALID;
  }
  const int64_t groups = (a.rows + rows_per_cta - 1) / rows_per_cta;
  if constexpr (MODE == ROW_MATVEC) {
    const size_t ssmem =
        row_staged_smem<T, NL>(pl.M, a.H, row_streams_multiplier<T, MCT>() ? 0 : rows_per_cta);
    if (ssmem <= 200 * 1024) {
      // persistent grid: as many CTAs as fit on the device at once (the
      // occupancy per device and staging size, kept per device)
      static std::atomic<unsigned long long> staged_mask{0};
      TRY_STATUS(ensure_dyn_smem(row_kernel_staged<T, NL, MCT>, 200 * 1024, staged_mask));
      struct Occ {
        size_t smem;
        int per_sm, sms;
      };
      static std::mutex occ_mutex;
      static Occ occ[64] = {};
      int dev = 0;
      GHB_CUDA_TRY(cudaGetDevice(&dev));
      Occ o{0, 0, 0};
      {
        std::lock_guard<std::mutex> lock(occ_mutex);
        if (dev < 64) o = occ[dev];
      }
      if (o.smem != ssmem) {
        o.smem = ssmem;
        GHB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, row_kernel_staged<T, NL, MCT>,
                                                                   row_threads<T, MCT>(), ssmem));
        GHB_CUDA_TRY(cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev));
        std::lock_guard<std::mutex> lock(occ_mutex);
        if (dev < 64) occ[dev] = o;
      }
      const int per_sm = o.per_sm, sms = o.sms;
      int64_t grid = static_cast<int64_t>(per_sm > 0 ? per_sm : 1) * sms;
      if (grid > groups) grid = groups;
      if (grid < 1) grid = 1;
      row_kernel_staged<T, NL, MCT><<<static_cast<unsigned>(grid), row_threads<T, MCT>(), ssmem, s>>>(a, pl,
                                                                                              rows_per_cta);
      GHB_CUDA_TRY(cudaGetLastError());
      return GHB_OK;
    }
  }
  int64_t grid = groups;
  if (MODE == ROW_ENERGY && grid > 1024) grid = 1024;   // partials hold 1024 x 6 doubles
  row_kernel<T, NL, MODE><<<static_cast<unsigned>(grid), kRowThreads, smem, s>>>(a, pl, rows_per_cta);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

// Size-specialised operator passes for one precision and transform length M
// (instantiated in the ct_*.cu units for FP32 and the ct64_*.cu units for FP64).
template <typename T, int M>
ghb_status launch_col_ct_m(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  constexpr int TW = col_tile_width(M, 2 * sizeof(T));
  return launch_col_tw<T, TW, M>(sign, mode, a, pl, s);
}
// Interleaved complex lines that give every thread a butterfly in every pass,
// for PER_ROW real lines per row (2 in 2-D, 3 in 3-D: a multiple of 3 so that
// the lines make whole rows), at most 32.
// In 3-D the counts below were chosen by a sweep of 6 .. 24 lines on GB300
// (one d = 3 operator application per setting): lines that make each pass
// about one full round of the block, with four FP32 CTAs per SM, beat the rule
// (M = 270: 12 lines, 221 against 242 us FP32 and 4.37 against 5.19 ms FP64;
// M = 162: 18 lines FP32, 55.8 against 61.7 us; M = 135: 12 lines FP32, 24 FP64;
// M = 72: 18 lines FP32).
template <typename T, int M, int PER_ROW>
__host__ __device__ constexpr int ct_fill_lines() {
  if (PER_ROW == 3) {
    if (M == 270) return 12;
    if (M == 162 && sizeof(T) == 4) return 18;
    if (M == 135) return sizeof(T) == 4 ? 12 : 24;
    if (M == 72 && sizeof(T) == 4) return 18;
  }
  constexpr int thr = row_threads<T, M>();
  int nl = (thr + ct_min_units<M>() - 1) / ct_min_units<M>();
  if (nl > 32) nl = 32;
  if (PER_ROW == 3) nl = 3 * ((nl + 2) / 3);
  if (nl > 32) nl = 30;
  return nl;
}

template <typename T, int M>
ghb_status launch_row_ct_m(int NL, const RowArgs& a, const FftPlan& pl, int rows_per_cta, cudaStream_t s) {
  // Short transforms (the 3-D double grids, 2-D ones up to M = 486) leave
  // most threads without a butterfly at one to three lines per CTA: take as
  // many rows as fill the CTA when the row rule leaves more than half of the
  // threads idle and the staging still fits (at M = 1458, where two lines
  // leave 44 % idle, four lines measured slower: 32.7 against 28.4 us).
  const int per_row = a.nfields * a.ncomp;
  constexpr int thr = row_threads<T, M>();
  if ((per_row == 2 || per_row == 3) && ct_min_units<M>() * NL * 2 < thr) {
    constexpr int NL2 = ct_fill_lines<T, M, 2>(), NL3 = ct_fill_lines<T, M, 3>();
    const int want = per_row == 2 ? NL2 : NL3;
    const int rows = 2 * want / per_row;
    const int arows = row_streams_multiplier<T, M>() ? 0 : rows;
    const size_t smem = per_row == 2 ? row_staged_smem<T, NL2>(M, a.H, arows) : row_staged_smem<T, NL3>(M, a.H, arows);
    if (want > NL && smem <= 200 * 1024) {
      if (per_row == 2) return launch_row_t<T, NL2, ROW_MATVEC, M>(a, pl, rows, s);
      return launch_row_t<T, NL3, ROW_MATVEC, M>(a, pl, rows, s);
    }
  }
  switch (NL) {
    case 1: return launch_row_t<T, 1, ROW_MATVEC, M>(a, pl, rows_per_cta, s);
    case 2: return launch_row_t<T, 2, ROW_MATVEC, M>(a, pl, rows_per_cta, s);
    case 3: return launch_row_t<T, 3, ROW_MATVEC, M>(a, pl, rows_per_cta, s);
    default: break;
  }
  set_error("internal: unsupported row-pass line count");
  return GHB_ERR_INVALID;
}

}  // namespace ghb
