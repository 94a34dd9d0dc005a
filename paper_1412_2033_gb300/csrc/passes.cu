// Transform passes of the double-grid Ga operator (Algorithm 2 on the Fourier
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
#include <algorithm>
#include <atomic>
#include <cmath>

#include "ghb_internal.cuh"

namespace ghb {

// Launchers defined by instantiation in the col_*.cu / row_*.cu units.
template <typename T, int TW, int MCT = 0>
ghb_status launch_col_tw(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s);
template <typename T, int NL, int MODE>
ghb_status launch_row_nl(const RowArgs& a, const FftPlan& pl, int rows_per_cta, cudaStream_t s);
template <typename T, int TW>
ghb_status launch_col_batch_tw(int sign, int mode, const ColItem* items, int n, int64_t blocks, size_t smem, int threads,
                               cudaStream_t s);
template <typename T, int NL, int MODE>
ghb_status launch_row_batch_nl(const RowItem* items, int n, int64_t blocks, size_t smem, int threads, cudaStream_t s);

template <typename T, int M>
ghb_status launch_col_ct_m(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s);
template <typename T, int M>
ghb_status launch_row_ct_m(int NL, const RowArgs& a, const FftPlan& pl, int rows_per_cta, cudaStream_t s);

template <typename T>
ghb_status launch_col_ct(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  switch (pl.M) {
    case 162: return launch_col_ct_m<T, 162>(sign, mode, a, pl, s);
    case 486: return launch_col_ct_m<T, 486>(sign, mode, a, pl, s);
    case 1458: return launch_col_ct_m<T, 1458>(sign, mode, a, pl, s);
    case 4374: return launch_col_ct_m<T, 4374>(sign, mode, a, pl, s);
    case 2187: return launch_col_ct_m<T, 2187>(sign, mode, a, pl, s);
    case 72: return launch_col_ct_m<T, 72>(sign, mode, a, pl, s);
    case 135: return launch_col_ct_m<T, 135>(sign, mode, a, pl, s);
    case 270: return launch_col_ct_m<T, 270>(sign, mode, a, pl, s);
    default: break;
  }
  set_error("internal: no size-specialised kernels for M=" + std::to_string(pl.M));
  return GHB_ERR_INVALID;
}
template ghb_status launch_col_ct<float>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);
template ghb_status launch_col_ct<double>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);

template <typename T>
ghb_status launch_row_ct(int NL, const RowArgs& a, const FftPlan& pl, int rows_per_cta, cudaStream_t s) {
  switch (pl.M) {
    case 162: return launch_row_ct_m<T, 162>(NL, a, pl, rows_per_cta, s);
    case 486: return launch_row_ct_m<T, 486>(NL, a, pl, rows_per_cta, s);
    case 1458: return launch_row_ct_m<T, 1458>(NL, a, pl, rows_per_cta, s);
    case 4374: return launch_row_ct_m<T, 4374>(NL, a, pl, rows_per_cta, s);
    case 2187: return launch_row_ct_m<T, 2187>(NL, a, pl, rows_per_cta, s);
    case 72: return launch_row_ct_m<T, 72>(NL, a, pl, rows_per_cta, s);
    case 135: return launch_row_ct_m<T, 135>(NL, a, pl, rows_per_cta, s);
    case 270: return launch_row_ct_m<T, 270>(NL, a, pl, rows_per_cta, s);
    default: break;
  }
  set_error("internal: no size-specialised kernels for M=" + std::to_string(pl.M));
  return GHB_ERR_INVALID;
}
template ghb_status launch_row_ct<float>(int, const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_ct<double>(int, const RowArgs&, const FftPlan&, int, cudaStream_t);

// The size-specialised kernels run where they are compiled and the plan
// carries their input order; FP32 follows the autotuner's choice, FP64 always
// takes them (its passes are bound by the FP64 pipe, where the compile-time
// roots save the most).
template <typename T>
bool use_ct(const FftPlan& pl, bool tuned_on) {
  if (pl.perm_ct == nullptr || !ct_size(pl.M)) return false;
  return sizeof(T) == 8 || tuned_on;
}

// Columns per CTA of a runtime-plan column pass over `outer` x `inner` lines:
// the widest tile (coalesced rows of up to 16 entries) whose CTAs still fill
// the device three times over; operands too narrow for that take the tile
// with the most CTAs.  Wide operands (the axis-1 pass in 3-D) get wide tiles,
// narrow ones (2-D operands of small N) narrow ones.
int auto_tile(int M, int64_t outer, int64_t inner, int elem_bytes) {
  static std::atomic<int> sms_cache{0};   // SM count (one device model per process)
  int sms = sms_cache.load(std::memory_order_relaxed);
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 152;
    sms_cache.store(sms, std::memory_order_relaxed);
  }
  int fallback = 0;
  for (int tw : {16, 8, 4, 2, 1}) {
    const size_t smem = col_smem_bytes(M, tw, elem_bytes);
    if (smem > 220 * 1024) continue;
    const int64_t per_sm = std::max<int64_t>(1, std::min<int64_t>(4, (227 * 1024) / static_cast<int64_t>(smem)));
    const int64_t ctas = outer * ((inner + tw - 1) / tw);
    if (ctas >= 3 * per_sm * sms) return tw;
    fallback = tw;   // the narrowest fitting tile: the most CTAs
  }
  return fallback > 0 ? fallback : 1;
}

template <typename T>
ghb_status launch_col(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  using C = typename CT<T>::type;
  if (use_ct<T>(pl, pl.ct_col != 0)) return launch_col_ct<T>(sign, mode, a, pl, s);
  const int forced = pl.tile[sizeof(T) == 4 ? 1 : 0];   // ghb_tune_set; 0 = by the operand
  const int TW = forced > 0 ? forced : auto_tile(pl.M, a.outer, a.inner, sizeof(C));
  if (col_smem_bytes(pl.M, TW, sizeof(C)) > 220 * 1024) {
    set_error("transform length too large for one CTA: M=" + std::to_string(pl.M));
    return GHB_ERR_INVALID;
  }
  switch (TW) {
    case 1: return launch_col_tw<T, 1>(sign, mode, a, pl, s);
    case 2: return launch_col_tw<T, 2>(sign, mode, a, pl, s);
    case 4: return launch_col_tw<T, 4>(sign, mode, a, pl, s);
    case 8: return launch_col_tw<T, 8>(sign, mode, a, pl, s);
    case 16: return launch_col_tw<T, 16>(sign, mode, a, pl, s);
    default: break;
  }
  set_error("internal: bad tile width");
  return GHB_ERR_INVALID;
}

template ghb_status launch_col<double>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);
template ghb_status launch_col<float>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);

// Rows a CTA transforms together in the operator's last-axis pass (d = 2:
// 1 or 2, the tuned value or by size: two rows for M <= 2048, one above; odd
// line counts always pair two rows).
void row_lines(int mode, int nfields, int ncomp, int M, int rows32, int* rows_per_cta, int* NL) {
  const int per_row = nfields * ncomp;
  int r = 1;
  if (mode == ROW_MATVEC || mode == ROW_TOREAL) r = (per_row % 2 == 1) ? 2 : 1;
  if (mode == ROW_MATVEC && per_row == 2) r = (rows32 == 1 || rows32 == 2) ? rows32 : (M <= 2048 ? 2 : 1);
  *rows_per_cta = r;
  *NL = (r * per_row + 1) / 2;
}

template <typename T>
ghb_status launch_col_batch(int sign, int mode, int TW, const ColItem* items, int n, int64_t blocks,
                            size_t smem, int threads, cudaStream_t s) {
  switch (TW) {
    case 1: return launch_col_batch_tw<T, 1>(sign, mode, items, n, blocks, smem, threads, s);
    case 2: return launch_col_batch_tw<T, 2>(sign, mode, items, n, blocks, smem, threads, s);
    case 4: return launch_col_batch_tw<T, 4>(sign, mode, items, n, blocks, smem, threads, s);
    case 8: return launch_col_batch_tw<T, 8>(sign, mode, items, n, blocks, smem, threads, s);
    case 16: return launch_col_batch_tw<T, 16>(sign, mode, items, n, blocks, smem, threads, s);
    default: break;
  }
  set_error("internal: bad tile width");
  return GHB_ERR_INVALID;
}
template ghb_status launch_col_batch<double>(int, int, int, const ColItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_col_batch<float>(int, int, int, const ColItem*, int, int64_t, size_t, int, cudaStream_t);

template <typename T>
ghb_status launch_row_batch(int mode, int NL, const RowItem* items, int n, int64_t blocks, size_t smem, int threads,
                            cudaStream_t s) {
  if (mode == ROW_MATVEC) {
    if (NL == 1) return launch_row_batch_nl<T, 1, ROW_MATVEC>(items, n, blocks, smem, threads, s);
    if (NL == 2) return launch_row_batch_nl<T, 2, ROW_MATVEC>(items, n, blocks, smem, threads, s);
    if (NL == 3) return launch_row_batch_nl<T, 3, ROW_MATVEC>(items, n, blocks, smem, threads, s);
  } else if constexpr (sizeof(T) == 8) {
    if (mode == ROW_TOREAL && NL == 1) return launch_row_batch_nl<T, 1, ROW_TOREAL>(items, n, blocks, smem, threads, s);
    if (mode == ROW_ENERGY) {
      switch (NL) {
        case 1: return launch_row_batch_nl<T, 1, ROW_ENERGY>(items, n, blocks, smem, threads, s);
        case 2: return launch_row_batch_nl<T, 2, ROW_ENERGY>(items, n, blocks, smem, threads, s);
        case 3: return launch_row_batch_nl<T, 3, ROW_ENERGY>(items, n, blocks, smem, threads, s);
        case 4: return launch_row_batch_nl<T, 4, ROW_ENERGY>(items, n, blocks, smem, threads, s);
        case 5: return launch_row_batch_nl<T, 5, ROW_ENERGY>(items, n, blocks, smem, threads, s);
        default: break;
      }
    }
  }
  set_error("internal: unsupported batched row pass");
  return GHB_ERR_INVALID;
}
template ghb_status launch_row_batch<double>(int, int, const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch<float>(int, int, const RowItem*, int, int64_t, size_t, int, cudaStream_t);

template <typename T>
ghb_status launch_row(int mode, const RowArgs& a, const FftPlan& pl, cudaStream_t s) {
  int rows_per_cta = 1, NL = 1;
  row_lines(mode, a.nfields, a.ncomp, pl.M, sizeof(T) == 4 ? pl.rows32 : 0, &rows_per_cta, &NL);
  if (mode == ROW_MATVEC) {
    if (use_ct<T>(pl, pl.ct_row != 0)) return launch_row_ct<T>(NL, a, pl, rows_per_cta, s);
    switch (NL) {
      case 1: return launch_row_nl<T, 1, ROW_MATVEC>(a, pl, rows_per_cta, s);
      case 2: return launch_row_nl<T, 2, ROW_MATVEC>(a, pl, rows_per_cta, s);
      case 3: return launch_row_nl<T, 3, ROW_MATVEC>(a, pl, rows_per_cta, s);
      default: break;
    }
  } else if constexpr (sizeof(T) == 8) {   // set-up and Gram passes run in FP64 only
    if (mode == ROW_TOREAL) {
      if (NL == 1) return launch_row_nl<T, 1, ROW_TOREAL>(a, pl, rows_per_cta, s);
      set_error("internal: unsupported row-pass line count");
      return GHB_ERR_INVALID;
    }
    switch (NL) {
      case 1: return launch_row_nl<T, 1, ROW_ENERGY>(a, pl, 1, s);
      case 2: return launch_row_nl<T, 2, ROW_ENERGY>(a, pl, 1, s);
      case 3: return launch_row_nl<T, 3, ROW_ENERGY>(a, pl, 1, s);
      case 4: return launch_row_nl<T, 4, ROW_ENERGY>(a, pl, 1, s);
      case 5: return launch_row_nl<T, 5, ROW_ENERGY>(a, pl, 1, s);
      default: break;
    }
  }
  set_error("internal: unsupported row-pass line count");
  return GHB_ERR_INVALID;
}

template ghb_status launch_row<double>(int, const RowArgs&, const FftPlan&, cudaStream_t);
template ghb_status launch_row<float>(int, const RowArgs&, const FftPlan&, cudaStream_t);

}  // namespace ghb
