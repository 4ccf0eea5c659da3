// logm_large_sqrt.cu -- instantiation of the whole-GPU kernel (logm_large.cuh): kModeSqrt, kModeSqrt with tensor-core updates.
#include "logm_large.cuh"

namespace lg {
namespace large_detail {
template cudaError_t launch_large_mode<kModeSqrt, false>(const SmallParams&, char*, cudaStream_t);
template cudaError_t launch_large_mode<kModeSqrt, true>(const SmallParams&, char*, cudaStream_t);
}  // namespace large_detail
}  // namespace lg
