// Instantiations of the last-axis pass kernels, FP64 (see passes_impl.cuh).
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

template ghb_status launch_row_nl<double, 1, ROW_MATVEC>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 2, ROW_MATVEC>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 3, ROW_MATVEC>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 1, ROW_TOREAL>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 1, ROW_ENERGY>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 2, ROW_ENERGY>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 3, ROW_ENERGY>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 4, ROW_ENERGY>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_nl<double, 5, ROW_ENERGY>(const RowArgs&, const FftPlan&, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 1, ROW_MATVEC>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 2, ROW_MATVEC>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 3, ROW_MATVEC>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 1, ROW_TOREAL>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 1, ROW_ENERGY>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 2, ROW_ENERGY>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 3, ROW_ENERGY>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 4, ROW_ENERGY>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_row_batch_nl<double, 5, ROW_ENERGY>(const RowItem*, int, int64_t, size_t, int, cudaStream_t);

}  // namespace ghb
