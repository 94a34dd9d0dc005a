// Size-specialised FP32 operator passes for the transform length M = 135
// (a double grid of the 3-D operator; see fft_ct.cuh and passes_impl.cuh).
#include "passes_impl.cuh"

namespace ghb {

template ghb_status launch_col_ct_m<float, 135>(int, int, const ColArgs&, const FftPlan&, cudaStream_t);
template ghb_status launch_row_ct_m<float, 135>(int, const RowArgs&, const FftPlan&, int, cudaStream_t);

}  // namespace ghb
