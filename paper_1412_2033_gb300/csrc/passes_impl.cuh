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

#include <cmath>

#include "ghb_internal.cuh"
#include "reduce.cuh"

namespace ghb {

// ---------------------------------------------------------------------------
// column pass: block `bid` of one operand handles tile (o, j0..j0+TW)
// ---------------------------------------------------------------------------
template <typename T, int TW, int SIGN, int MODE>
__device__ __forceinline__ void col_body(const ColArgs& a, const FftPlan& pl, int64_t bid) {
  using C = typename CT<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  __shared__ PassSmem st;
  if (a.st != nullptr && a.st->done != RUNNING) return;
  const int npass = load_passes<C>(st, pl);

  const int M = pl.M;
  const int64_t tiles = (a.inner + TW - 1) / TW;
  const int64_t o = bid / tiles;
  const int64_t j0 = (bid % tiles) * TW;
  const int width = static_cast<int>(a.inner - j0 < TW ? a.inner - j0 : TW);
  const C* __restrict__ tw = twtab<C>(pl);
  const int* __restrict__ perm = pl.perm;

  if (SIGN > 0) {
    for (int u = threadIdx.x; u < static_cast<int>(padded_elems<C>(M * TW)); u += blockDim.x) buf[u] = mk(T(0), T(0));
    __syncthreads();
    const C* __restrict__ in = static_cast<const C*>(a.in);
    const int Lin = a.Lin;
    const int half = (Lin - 1) / 2;
    T beta = T(0);
    if (MODE == COL_PUPDATE) beta = static_cast<T>(a.st->beta);
    for (int u = threadIdx.x; u < Lin * TW; u += blockDim.x) {
      const int t = u % TW;
      const int i = u / TW;
      if (t < width) {
        const int64_t idx = (o * Lin + i) * a.inner + j0 + t;
        C v = in[idx];
        if (MODE == COL_PUPDATE) {
          C po = static_cast<const C*>(a.pold)[idx];
          v = mk(v.x + beta * po.x, v.y + beta * po.y);
          static_cast<C*>(a.pnew)[idx] = v;
        }
        int k = i - half;
        if (k < 0) k += M;
        buf[pidx<C>(__ldg(&perm[k]) * TW + t)] = v;
      }
    }
    __syncthreads();
    fft_dit<+1, TW>(buf, st, npass, M, tw, roottab<C>(pl));
    C* __restrict__ out = static_cast<C*>(a.out);
    for (int u = threadIdx.x; u < M * TW; u += blockDim.x) {
      const int t = u % TW;
      const int m = u / TW;
      if (t < width) out[(o * M + m) * a.inner + j0 + t] = buf[pidx<C>(m * TW + t)];
    }
  } else {
    const C* __restrict__ in = static_cast<const C*>(a.in);
    for (int u = threadIdx.x; u < M * TW; u += blockDim.x) {
      const int t = u % TW;
      const int m = u / TW;
      buf[pidx<C>(u)] = (t < width) ? in[(o * M + m) * a.inner + j0 + t] : mk(T(0), T(0));
    }
    __syncthreads();
    fft_dif<-1, TW>(buf, st, npass, M, tw, roottab<C>(pl));
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
        C v = buf[pidx<C>(__ldg(&perm[k]) * TW + t)];
        out[(o * Lout + i) * a.inner + j0 + t] = inv * v;
      }
    }
  }
}


constexpr int kColThreads32 = 512;
constexpr int kColThreads64 = 256;

template <typename T, int TW, int SIGN, int MODE>
__global__ void __launch_bounds__(sizeof(T) == 8 ? kColThreads64 : kColThreads32)
    col_kernel(ColArgs a, FftPlan pl) {
  col_body<T, TW, SIGN, MODE>(a, pl, blockIdx.x);
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

template <typename T, int TW, int SIGN, int MODE>
inline ghb_status launch_col_t(const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  using C = typename CT<T>::type;
  const size_t smem = col_smem_bytes(pl.M, TW, sizeof(C));
  static bool attr_set = false;
  if (!attr_set) {
    GHB_CUDA_TRY(cudaFuncSetAttribute(col_kernel<T, TW, SIGN, MODE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr_set = true;
  }
  const int64_t tiles = (a.inner + TW - 1) / TW;
  const int64_t grid = tiles * a.outer;
  const int threads = (sizeof(T) == 4 && pl.M * TW >= 2048) ? kColThreads32 : 256;
  col_kernel<T, TW, SIGN, MODE><<<static_cast<unsigned>(grid), threads, smem, s>>>(a, pl);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

// All sign/mode variants of one precision and tile width.
template <typename T, int TW>
ghb_status launch_col_tw(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  if (sign > 0)
    return mode == COL_PUPDATE ? launch_col_t<T, TW, +1, COL_PUPDATE>(a, pl, s)
                               : launch_col_t<T, TW, +1, COL_PLAIN>(a, pl, s);
  return launch_col_t<T, TW, -1, COL_PLAIN>(a, pl, s);
}

template <typename T, int TW, int SIGN, int MODE>
inline ghb_status launch_col_batch_t(const ColItem* items, int n, int64_t blocks, size_t smem,
                                     cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    GHB_CUDA_TRY(cudaFuncSetAttribute(col_kernel_batch<T, TW, SIGN, MODE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr_set = true;
  }
  const int threads = sizeof(T) == 4 ? kColThreads32 : kColThreads64;
  col_kernel_batch<T, TW, SIGN, MODE><<<static_cast<unsigned>(blocks), threads, smem, s>>>(items, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

template <typename T, int TW>
ghb_status launch_col_batch_tw(int sign, int mode, const ColItem* items, int n, int64_t blocks, size_t smem,
                               cudaStream_t s) {
  if (sign > 0)
    return mode == COL_PUPDATE ? launch_col_batch_t<T, TW, +1, COL_PUPDATE>(items, n, blocks, smem, s)
                               : launch_col_batch_t<T, TW, +1, COL_PLAIN>(items, n, blocks, smem, s);
  return launch_col_batch_t<T, TW, -1, COL_PLAIN>(items, n, blocks, smem, s);
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
        A = static_cast<const C*>(a.t[d0.field])[d0.comp * a.comp_stride + d0.row * H + k];
      if (d1.valid)
        B = static_cast<const C*>(a.t[d1.field])[d1.comp * a.comp_stride + d1.row * H + k];
      buf[pidx<C>(__ldg(&perm[k]) * NL + j)] = mk(A.x - B.y, A.y + B.x);
      if (k > 0) buf[pidx<C>(__ldg(&perm[M - k]) * NL + j)] = mk(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    fft_dit<+1, NL>(buf, st, npass, M, tw, roottab<C>(pl));

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
      fft_dif<-1, NL>(buf, st, npass, M, tw, roottab<C>(pl));
      const T sc = T(0.5) / T(M);
      for (int u = threadIdx.x; u < NL * H; u += blockDim.x) {
        const int j = (NL == 1) ? 0 : u % NL;
        const int k = (NL == 1) ? u : u / NL;
        const LineDesc d0 = ld[2 * j], d1 = ld[2 * j + 1];
        const C W = buf[pidx<C>(__ldg(&perm[k]) * NL + j)];
        const C Wm = buf[pidx<C>(__ldg(&perm[k == 0 ? 0 : M - k]) * NL + j)];
        if (d0.valid)
          static_cast<C*>(a.t[d0.field])[d0.comp * a.comp_stride + d0.row * H + k] =
              mk(sc * (W.x + Wm.x), sc * (W.y - Wm.y));
        if (d1.valid)
          static_cast<C*>(a.t[d1.field])[d1.comp * a.comp_stride + d1.row * H + k] =
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

template <typename T, int NL, int MODE>
__global__ void __launch_bounds__(kRowThreads) row_kernel(RowArgs a, FftPlan pl, int rows_per_cta) {
  row_body<T, NL, MODE>(a, pl, rows_per_cta, blockIdx.x, gridDim.x);
}

template <typename T, int NL, int MODE>
__global__ void __launch_bounds__(kRowThreads) row_kernel_batch(const RowItem* __restrict__ items, int n) {
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = find_item(items, n, blockIdx.x);
  __syncthreads();
  const RowItem& it = items[s_item];
  row_body<T, NL, MODE>(it.a, *it.pl, it.rows_per_cta, blockIdx.x - it.block_begin, it.nblocks);
}

template <typename T, int NL, int MODE>
inline ghb_status launch_row_batch_t(const RowItem* items, int n, int64_t blocks, size_t smem,
                                     cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    GHB_CUDA_TRY(cudaFuncSetAttribute(row_kernel_batch<T, NL, MODE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  row_kernel_batch<T, NL, MODE><<<static_cast<unsigned>(blocks), kRowThreads, smem, s>>>(items, n);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

template <typename T, int NL, int MODE>
inline ghb_status launch_row_t(const RowArgs& a, const FftPlan& pl, int rows_per_cta,
                               cudaStream_t s) {
  using C = typename CT<T>::type;
  const size_t smem = padded_elems<C>(static_cast<size_t>(pl.M) * NL) * sizeof(C);
  static bool attr_set = false;
  if (!attr_set) {
    GHB_CUDA_TRY(cudaFuncSetAttribute(row_kernel<T, NL, MODE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  if (smem > 200 * 1024) {
    set_error("row transform too large for one CTA: M=" + std::to_string(pl.M));
    return GHB_ERR_INVALID;
  }
  const int64_t groups = (a.rows + rows_per_cta - 1) / rows_per_cta;
  int64_t grid = groups;
  if (MODE == ROW_ENERGY && grid > 1024) grid = 1024;   // partials hold 1024 x 6 doubles
  row_kernel<T, NL, MODE><<<static_cast<unsigned>(grid), kRowThreads, smem, s>>>(a, pl, rows_per_cta);
  GHB_CUDA_TRY(cudaGetLastError());
  return GHB_OK;
}

}  // namespace ghb
