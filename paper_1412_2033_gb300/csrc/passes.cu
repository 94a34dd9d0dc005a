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
#include <cmath>

#include "ghb_internal.cuh"

namespace ghb {

size_t col_smem_bytes(int M, int TW, int elem_bytes) {
  return elem_bytes == 8 ? padded_elems<float2>(static_cast<size_t>(M) * TW) * 8
                         : padded_elems<double2>(static_cast<size_t>(M) * TW) * 16;
}

// Widest tile that keeps two CTAs per SM (<= ~110 KB of shared memory).
int col_tile_width(int M, int elem_bytes) {
  const size_t budget = 110 * 1024;
  for (int tw : {16, 8, 4, 2}) {
    if (col_smem_bytes(M, tw, elem_bytes) <= budget) return tw;
  }
  return 1;
}

// Launchers defined by instantiation in the col_*.cu / row_*.cu units.
template <typename T, int TW>
ghb_status launch_col_tw(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s);
template <typename T, int NL, int MODE>
ghb_status launch_row_nl(const RowArgs& a, const FftPlan& pl, int rows_per_cta, cudaStream_t s);
template <typename T, int TW>
ghb_status launch_col_batch_tw(int sign, int mode, const ColItem* items, int n, int64_t blocks, size_t smem,
                               cudaStream_t s);
template <typename T, int NL, int MODE>
ghb_status launch_row_batch_nl(const RowItem* items, int n, int64_t blocks, size_t smem, cudaStream_t s);

template <typename T>
ghb_status launch_col(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s) {
  using C = typename CT<T>::type;
  const int TW = col_tile_width(pl.M, sizeof(C));
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

void row_lines(int mode, int nfields, int ncomp, int* rows_per_cta, int* NL) {
  const int per_row = nfields * ncomp;
  int r = 1;
  if (mode == ROW_MATVEC || mode == ROW_TOREAL) r = (per_row % 2 == 1) ? 2 : 1;
  *rows_per_cta = r;
  *NL = (r * per_row + 1) / 2;
}

template <typename T>
ghb_status launch_col_batch(int sign, int mode, int TW, const ColItem* items, int n, int64_t blocks,
                            size_t smem, cudaStream_t s) {
  switch (TW) {
    case 1: return launch_col_batch_tw<T, 1>(sign, mode, items, n, blocks, smem, s);
    case 2: return launch_col_batch_tw<T, 2>(sign, mode, items, n, blocks, smem, s);
    case 4: return launch_col_batch_tw<T, 4>(sign, mode, items, n, blocks, smem, s);
    case 8: return launch_col_batch_tw<T, 8>(sign, mode, items, n, blocks, smem, s);
    case 16: return launch_col_batch_tw<T, 16>(sign, mode, items, n, blocks, smem, s);
    default: break;
  }
  set_error("internal: bad tile width");
  return GHB_ERR_INVALID;
}
template ghb_status launch_col_batch<double>(int, int, int, const ColItem*, int, int64_t, size_t, cudaStream_t);
template ghb_status launch_col_batch<float>(int, int, int, const ColItem*, int, int64_t, size_t, cudaStream_t);

template <typename T>
ghb_status launch_row_batch(int mode, int NL, const RowItem* items, int n, int64_t blocks, size_t smem,
                            cudaStream_t s) {
  if (mode == ROW_MATVEC) {
    if (NL == 1) return launch_row_batch_nl<T, 1, ROW_MATVEC>(items, n, blocks, smem, s);
    if (NL == 3) return launch_row_batch_nl<T, 3, ROW_MATVEC>(items, n, blocks, smem, s);
  } else if constexpr (sizeof(T) == 8) {
    if (mode == ROW_TOREAL && NL == 1) return launch_row_batch_nl<T, 1, ROW_TOREAL>(items, n, blocks, smem, s);
    if (mode == ROW_ENERGY) {
      switch (NL) {
        case 1: return launch_row_batch_nl<T, 1, ROW_ENERGY>(items, n, blocks, smem, s);
        case 2: return launch_row_batch_nl<T, 2, ROW_ENERGY>(items, n, blocks, smem, s);
        case 3: return launch_row_batch_nl<T, 3, ROW_ENERGY>(items, n, blocks, smem, s);
        case 4: return launch_row_batch_nl<T, 4, ROW_ENERGY>(items, n, blocks, smem, s);
        case 5: return launch_row_batch_nl<T, 5, ROW_ENERGY>(items, n, blocks, smem, s);
        default: break;
      }
    }
  }
  set_error("internal: unsupported batched row pass");
  return GHB_ERR_INVALID;
}
template ghb_status launch_row_batch<double>(int, int, const RowItem*, int, int64_t, size_t, cudaStream_t);
template ghb_status launch_row_batch<float>(int, int, const RowItem*, int, int64_t, size_t, cudaStream_t);

template <typename T>
ghb_status launch_row(int mode, const RowArgs& a, const FftPlan& pl, cudaStream_t s) {
  int rows_per_cta = 1, NL = 1;
  row_lines(mode, a.nfields, a.ncomp, &rows_per_cta, &NL);
  if (mode == ROW_MATVEC) {
    switch (NL) {
      case 1: return launch_row_nl<T, 1, ROW_MATVEC>(a, pl, rows_per_cta, s);
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
