// logm_large_exec_tc.cu -- instantiation of the whole-GPU kernel (logm_large.cuh): kModeExecute with tensor-core updates.
#include "logm_large.cuh"

namespace lg {
namespace large_detail {
template cudaError_t launch_large_mode<kModeExecute, true>(const SmallParams&, char*, cudaStream_t);
}  // namespace large_detail
}  // namespace lg
