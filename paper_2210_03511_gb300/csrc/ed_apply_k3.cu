// H.x kernels for value kind 3 (complex FP32 vectors).
#include "ed_apply_impl.cuh"

namespace ed {
template ed_status apply_launch_kind<3>(const HxArgs&, size_t, int, bool, bool, bool, cudaStream_t);
template ed_status apply_batch_kind<3>(const BatchLaunch&, cudaStream_t);
}  // namespace ed
