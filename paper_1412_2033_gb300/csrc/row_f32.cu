// Instantiations of the last-axis pass kernels, FP32 (see passes_impl.cuh).
#include "passes_impl.cuh"

namespace ghb {

template <typename T, int NL, int MODE>
ghb_status launch_row_nl(const RowArgs& a, const FftPlan& pl, int rows_per_cta, cudaStream_t s) {
  return launch_row_t<T, NL, MODE>(a, pl, rows_per_cta, s);
}

template <typename T, int NL, int MODE>
ghb_status launch_row_batch_nl(const RowItem* items, int n, int64_t blocks, size_t smem, int threads, cudaStream_t s) {
  return launch_row_batch_t<T, NL, MODE>(items, n, blocks, smem, threads, s);
}

template ghb_status launch_row_nl<float, 1, ROW_MATVEC>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<float, 2, ROW_MATVEC>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<float, 3, ROW_MATVEC>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_batch_nl<float, 1, ROW_MATVEC>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<float, 2, ROW_MATVEC>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<float, 3, ROW_MATVEC>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);

}  // namespace ghb
