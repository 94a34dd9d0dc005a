// Instantiations of the transform-pass kernels (see passes_impl.cuh).
#include "passes_impl.cuh"

namespace ghb {

template ghb_status launch_col_tw<float, 1>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);
template ghb_status launch_col_tw<float, 2>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);
template ghb_status launch_col_tw<float, 4>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);

template ghb_status launch_col_batch_tw<float, 1>(int, int, const ColItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_col_batch_tw<float, 2>(int, int, const ColItem*, int, int64_t, size_t, int, cudaStream_t);
template ghb_status launch_col_batch_tw<float, 4>(int, int, const ColItem*, int, int64_t, size_t, int, cudaStream_t);

}  // namespace ghb
