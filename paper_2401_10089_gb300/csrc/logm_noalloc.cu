// logm_noalloc.cu -- logm_execute for callers that cannot allocate device
// memory themselves.
//
// Some callers have no way to obtain a device buffer for the workspace: code
// that runs inside a framework or plugin host that owns every device
// allocation, real-time or embedded callers with a fixed device-memory budget
// set at start-up, and host code that may not call cudaMalloc at the point
// where it needs the logarithm. For them this file keeps the scratch space
// the one-block-per-matrix kernel needs in a fixed file-scope device array,
// so the call takes only the caller's inputs and outputs.
//
// The array is kNoallocScratchBytes (32 MiB) and every GPU that loads the
// library keeps it until the process exits. The call uses as many
// one-matrix workspace slots as fit in it (each slot is 7 n_max^2 doubles),
// so it runs fewer matrices at a time than logm_execute when n_max is large.
#include <mutex>

#include "../../include/logm.h"
#include "logm_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// The scratch array. Host code must not pass `g_noalloc_scratch` itself to a
// kernel: on the host that name is a stand-in, not a device address. The
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Set-up, once per device, with that device current: look up the device
// address of the scratch array. Returns LOGM_SUCCESS or an error code.
int scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LOGM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LOGM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return LOGM_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LOGM_SUCCESS;
}

}  // namespace

extern "C" int logm_execute_noalloc(const logm_batch* batch, const logm_options* opts,
                                    const void* A, void* L, int32_t* s_dev, int32_t* k_dev,
                                    int32_t* info_dev, void* stream) {
  if (!batch || !opts) return LOGM_ERR_INVALID_ARG;
  if (batch->count < 0) return LOGM_ERR_INVALID_ARG;
  if (batch->dtype != LOGM_DTYPE_F64 && batch->dtype != LOGM_DTYPE_F32) return LOGM_ERR_INVALID_ARG;
  int n_max = batch->n_uniform;
  if (n_max <= 0) {
    if (batch->n_max <= 0 || (batch->count > 0 && (!batch->n || !batch->offset)))
      return LOGM_ERR_INVALID_ARG;
    n_max = batch->n_max;
  }
  if (opts->k_max < 1 || opts->k_max > 6) return LOGM_ERR_INVALID_ARG;
  if (opts->max_sqrt < 0 || opts->max_sqrt > 1000) return LOGM_ERR_INVALID_ARG;
  if (opts->max_db_iter < 1 || opts->max_db_iter > 1000) return LOGM_ERR_INVALID_ARG;
  if (opts->db_form != LOGM_DB_TWO_INVERSE && opts->db_form != LOGM_DB_PRODUCT) return LOGM_ERR_INVALID_ARG;
  if (opts->balance != LOGM_BALANCE_NONE && opts->balance != LOGM_BALANCE_SCALE) return LOGM_ERR_INVALID_ARG;
  if (opts->fp64_products != LOGM_FP64_PIPE && opts->fp64_products != LOGM_FP64_TC_SLICED) return LOGM_ERR_INVALID_ARG;
  for (int t = 0; t < 5; ++t)
    if (!(opts->theta[t] >= 0.0) || !(opts->theta[t] < 1.0)) return LOGM_ERR_INVALID_ARG;
  if (opts->precision != LOGM_PREC_FP64) return LOGM_ERR_UNSUPPORTED;
  // Balancing keeps diag(T) per matrix (count * n_max doubles), which has no
  // fixed bound: not offered here.
  if (opts->balance != LOGM_BALANCE_NONE) return LOGM_ERR_UNSUPPORTED;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !L || !info_dev) return LOGM_ERR_INVALID_ARG;
  // Sizes beyond what this entry point can hold are rejected here.
  if (n_max > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
  const size_t slot_bytes = (size_t)lg::kSlotMats * (size_t)n_max * n_max * sizeof(double);
  const size_t fit = (kNoallocScratchBytes - 256) / slot_bytes;
  if (fit < 1) return LOGM_ERR_WORKSPACE;

  void* scratch = nullptr;
  if (int r = scratch_for_current_device(&scratch)) return r;

  lg::SmallParams p{};
  p.count = batch->count;
  p.dtype = batch->dtype;
  p.n_uniform = batch->n_uniform > 0 ? batch->n_uniform : 0;
  p.n_max = n_max;
  p.batch_nmax = n_max;
  p.n_dev = batch->n;
  p.off_dev = batch->offset;
  p.k_max = opts->k_max;
  p.max_sqrt = opts->max_sqrt;
  p.max_db = opts->max_db_iter;
  for (int t = 0; t < 5; ++t) p.theta[t] = opts->theta[t] > 0.0 ? opts->theta[t] : lg::kThetaPaper[t];
  p.precision = opts->precision;
  p.db_form = opts->db_form;
  p.A = A;
  p.L = L;
  p.s_out = s_dev;
  p.k_out = k_dev;
  p.info = info_dev;
  // First 256 bytes: the work-queue counter (launch_small zeroes it on the
  // stream before the kernel); then the slots, which need no clearing.
  p.queue = static_cast<int32_t*>(scratch);
  p.slots = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + 256);
  const int want = lg::small_kernel_slots(batch->count);
  p.n_slots = (size_t)want < fit ? want : (int)fit;
  const cudaError_t e = lg::launch_small(lg::kModeExecute, p, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LOGM_SUCCESS : LOGM_ERR_CUDA;
}
