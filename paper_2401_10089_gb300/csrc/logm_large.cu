// logm_large.cu -- dispatch of the whole-GPU kernel (logm_large.cuh) by
// mode and update path; the instantiations live in logm_large_*.cu.
#include "logm_large.cuh"

namespace lg {
namespace large_detail {
extern template cudaError_t launch_large_mode<kModeExecute, false>(const SmallParams&, char*, cudaStream_t);
extern template cudaError_t launch_large_mode<kModeExecute, true>(const SmallParams&, char*, cudaStream_t);
extern template cudaError_t launch_large_mode<kModePlan, false>(const SmallParams&, char*, cudaStream_t);
extern template cudaError_t launch_large_mode<kModeSqrt, false>(const SmallParams&, char*, cudaStream_t);
extern template cudaError_t launch_large_mode<kModeSqrt, true>(const SmallParams&, char*, cudaStream_t);
extern template cudaError_t launch_large_mode<kModeGraph, false>(const SmallParams&, char*, cudaStream_t);
}  // namespace large_detail

size_t large_workspace_bytes(int n_max) { return large_detail::large_layout(n_max).total; }

// Self-test of the grid barrier's bound: two co-resident blocks wait at a
// barrier for 2 + missing arrivals; with missing > 0 nobody completes it, so
// both give up after timeout_ns and the status word reads 1 (the whole-GPU
// kernel reports that as LOGM_INFO_TIMEOUT); with missing = 0 it reads 0.
__global__ void k_barrier_probe(unsigned long long* bar, int* status, unsigned nwait,
                                unsigned long long timeout_ns) {
  __shared__ unsigned long long ep;
  if (threadIdx.x == 0) ep = 0;
  __syncthreads();
  bounded_barrier(bar, nwait, status, &ep, timeout_ns);
}

cudaError_t launch_barrier_probe(int missing, unsigned long long timeout_ns, void* ws, cudaStream_t st) {
  unsigned long long* bar = static_cast<unsigned long long*>(ws);
  int* status = reinterpret_cast<int*>(static_cast<char*>(ws) + 8);
  cudaError_t e = cudaMemsetAsync(ws, 0, 16, st);
  if (e != cudaSuccess) return e;
  unsigned nwait = 2u + static_cast<unsigned>(missing);
  void* args[] = {&bar, &status, &nwait, &timeout_ns};
  return cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(2), dim3(32), args, 0, st);
}

cudaError_t launch_large(Mode mode, const SmallParams& p, void* ws, cudaStream_t st) {
  if (p.count <= 0) return cudaSuccess;
  char* w = static_cast<char*>(ws);
  const bool tc = p.fp64_tc != 0;
  switch (mode) {
    case kModeExecute:
      return tc ? large_detail::launch_large_mode<kModeExecute, true>(p, w, st) : large_detail::launch_large_mode<kModeExecute, false>(p, w, st);
    case kModePlan: return large_detail::launch_large_mode<kModePlan, false>(p, w, st);
    case kModeSqrt:
      return tc ? large_detail::launch_large_mode<kModeSqrt, true>(p, w, st) : large_detail::launch_large_mode<kModeSqrt, false>(p, w, st);
    case kModeGraph: return large_detail::launch_large_mode<kModeGraph, false>(p, w, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lg
