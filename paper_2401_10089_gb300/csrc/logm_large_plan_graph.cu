// logm_large_plan_graph.cu -- instantiation of the whole-GPU kernel (logm_large.cuh): kModePlan, kModeGraph.
#include "logm_large.cuh"

namespace lg {
namespace large_detail {
template cudaError_t launch_large_mode<kModePlan, false>(const SmallParams&, char*, cudaStream_t);
template cudaError_t launch_large_mode<kModeGraph, false>(const SmallParams&, char*, cudaStream_t);
}  // namespace large_detail
}  // namespace lg
