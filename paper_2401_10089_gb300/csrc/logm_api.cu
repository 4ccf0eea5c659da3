// logm_api.cu -- the extern "C" entry points declared in include/logm.h.
// Argument checking, workspace layout and dispatch; every step of the method
// runs in the kernels this file launches.
#include <cstdint>
#include <cstring>

#include "../../include/logm.h"
#include "logm_internal.h"

namespace {

constexpr double kThetaPaper[3] = {1.83e-8, 1.53e-4, 2.46e-1};  // Table Table_theta, k = 1, 2, 5

int batch_n_max(const logm_batch* b) {
  if (!b) return -1;
  if (b->count < 0) return -1;
  if (b->dtype != LOGM_DTYPE_F64 && b->dtype != LOGM_DTYPE_F32) return -1;
  if (b->n_uniform > 0) return b->n_uniform;
  if (b->n_max <= 0 || (b->count > 0 && (!b->n || !b->offset))) return -1;
  return b->n_max;
}

int opts_ok(const logm_options* o) {
  if (!o) return 0;
  if (o->k_max != 1 && o->k_max != 2 && o->k_max != 5) return 0;
  if (o->precision < LOGM_PREC_FP64 || o->precision > LOGM_PREC_BF16X3) return 0;
  if (o->max_sqrt < 0 || o->max_sqrt > 1000) return 0;
  if (o->max_db_iter < 1 || o->max_db_iter > 1000) return 0;
  for (int t = 0; t < 3; ++t)
    if (!(o->theta[t] >= 0.0) || !(o->theta[t] < 1.0)) return 0;
  return 1;
}

// Workspace: [small part | large part]. The small part (queue, order, one
// slot of kSlotMats matrices per resident block) serves matrices with
// n <= kSmallMaxN; the large part (one whole-GPU slot) serves n > kSmallMaxN.
struct WsLayout {
  int small_nmax;   // 0: no small pass
  int large_nmax;   // 0: no large pass
  size_t small_bytes, large_off, total;
};

WsLayout ws_layout(const logm_batch* b) {
  WsLayout L{};
  const int n_max = batch_n_max(b);
  if (n_max <= 0) return L;
  const bool ragged = b->n_uniform <= 0;
  if (n_max <= lg::kSmallMaxN) {
    L.small_nmax = n_max;
  } else {
    L.large_nmax = n_max;
    if (ragged) L.small_nmax = lg::kSmallMaxN;
  }
  L.small_bytes = L.small_nmax ? lg::small_workspace_bytes(b->count, L.small_nmax) : 0;
  L.large_off = (L.small_bytes + 255) / 256 * 256;
  L.total = L.large_off + (L.large_nmax ? lg::large_workspace_bytes(L.large_nmax) : 0);
  return L;
}

void fill_common(lg::SmallParams& p, const logm_batch* b, const logm_options* o) {
  std::memset(&p, 0, sizeof(p));
  p.count = b->count;
  p.dtype = b->dtype;
  p.n_uniform = b->n_uniform > 0 ? b->n_uniform : 0;
  p.n_max = batch_n_max(b);
  p.n_dev = b->n;
  p.off_dev = b->offset;
  if (o) {
    p.k_max = o->k_max;
    p.max_sqrt = o->max_sqrt;
    p.max_db = o->max_db_iter;
    for (int t = 0; t < 3; ++t) p.theta[t] = o->theta[t] > 0.0 ? o->theta[t] : kThetaPaper[t];
    p.precision = o->precision;
  } else {
    p.k_max = 5;
    p.max_sqrt = 40;
    p.max_db = 50;
    for (int t = 0; t < 3; ++t) p.theta[t] = kThetaPaper[t];
  }
  p.ctx_nmax = p.n_max;
}

// Launch the small pass and/or the large pass for this batch.
int run_passes(lg::Mode mode, lg::SmallParams& p, const logm_batch* b, void* ws, cudaStream_t st) {
  const WsLayout L = ws_layout(b);
  char* w = static_cast<char*>(ws);
  if (L.small_nmax) {
    lg::SmallParams q = p;
    q.n_max = L.small_nmax;
    q.large_pass = L.large_nmax ? 1 : 0;
    q.queue = reinterpret_cast<int32_t*>(w);
    const size_t ob = lg::small_order_bytes(b->count);
    q.order = reinterpret_cast<int32_t*>(w + 256);
    q.order_aux = q.order + b->count;
    q.slots = reinterpret_cast<double*>(w + 256 + ob);
    q.n_slots = lg::small_kernel_slots(b->count);
    if (lg::launch_small(mode, q, st) != cudaSuccess) return LOGM_ERR_CUDA;
  }
  if (L.large_nmax) {
    lg::SmallParams q = p;
    q.n_max = L.large_nmax;
    q.large_pass = L.small_nmax ? 1 : 0;
    if (lg::launch_large(mode, q, w + L.large_off, st) != cudaSuccess) return LOGM_ERR_CUDA;
  }
  return LOGM_SUCCESS;
}

int check_ws(const logm_batch* b, void* ws, size_t ws_bytes) {
  if (!ws) return LOGM_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return LOGM_ERR_WORKSPACE;
  if (ws_bytes < ws_layout(b).total) return LOGM_ERR_WORKSPACE;
  return LOGM_SUCCESS;
}

}  // namespace

extern "C" {

int logm_version(void) { return 100; }

size_t logm_workspace_size(const logm_batch* batch, const logm_options* opts) {
  (void)opts;
  if (batch_n_max(batch) <= 0) return 0;
  return ws_layout(batch).total;
}

size_t logm_context_size(const logm_batch* batch, const logm_options* opts) {
  (void)opts;
  const int n_max = batch_n_max(batch);
  if (n_max <= 0) return 0;
  return (size_t)batch->count * lg::kCtxLevels * (size_t)n_max * n_max * sizeof(double) + 256;
}

int logm_plan(const logm_batch* batch, const logm_options* opts, const void* A, const void* AI2,
              int32_t* finish_dev, int32_t* k_dev, double* alpha_dev, int32_t* info_dev, void* ws,
              size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !finish_dev || !k_dev || !alpha_dev || !info_dev) return LOGM_ERR_INVALID_ARG;
  if (int r = check_ws(batch, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, opts);
  p.A = A;
  p.AI2_in = AI2;
  p.finish = finish_dev;
  p.k_out = k_dev;
  p.alpha = alpha_dev;
  p.info = info_dev;
  return run_passes(lg::kModePlan, p, batch, ws, static_cast<cudaStream_t>(stream));
}

int logm_sqrt(const logm_batch* batch, const logm_options* opts, void* A, void* A2_out,
              void* AI2_out, const int32_t* active_dev, int32_t* iters_dev, int32_t* info_dev,
              void* ws, size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !info_dev) return LOGM_ERR_INVALID_ARG;
  if (int r = check_ws(batch, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, opts);
  p.A_inout = A;
  p.A2_out = A2_out;
  p.AI2_out = AI2_out;
  p.active = active_dev;
  p.iters = iters_dev;
  p.info = info_dev;
  return run_passes(lg::kModeSqrt, p, batch, ws, static_cast<cudaStream_t>(stream));
}

int logm_graph_eval(const logm_batch* batch, int32_t precision, const void* X, const void* P3,
                    const int32_t* k_dev, void* Z, void* ws, size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0) return LOGM_ERR_INVALID_ARG;
  if (precision < LOGM_PREC_FP64 || precision > LOGM_PREC_BF16X3) return LOGM_ERR_INVALID_ARG;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!X || !k_dev || !Z) return LOGM_ERR_INVALID_ARG;
  if (precision != LOGM_PREC_FP64) return LOGM_ERR_UNSUPPORTED;
  if (int r = check_ws(batch, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, nullptr);
  p.X = X;
  p.P3 = P3;
  p.k_in = k_dev;
  p.L = Z;
  p.precision = precision;
  return run_passes(lg::kModeGraph, p, batch, ws, static_cast<cudaStream_t>(stream));
}

int logm_execute(const logm_batch* batch, const logm_options* opts, const void* A, void* L,
                 int32_t* s_dev, int32_t* k_dev, int32_t* info_dev, int32_t* stats_dev, void* ctx,
                 void* ws, size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !L || !info_dev) return LOGM_ERR_INVALID_ARG;
  if (opts->precision != LOGM_PREC_FP64) return LOGM_ERR_UNSUPPORTED;
  if (int r = check_ws(batch, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, opts);
  p.A = A;
  p.L = L;
  p.s_out = s_dev;
  p.k_out = k_dev;
  p.info = info_dev;
  p.stats = stats_dev;
  p.ctx = static_cast<double*>(ctx);
  p.ctx_levels = lg::kCtxLevels;
  return run_passes(lg::kModeExecute, p, batch, ws, static_cast<cudaStream_t>(stream));
}

int logm_backward(const logm_batch* batch, const logm_options* opts, const void* A, const void* ctx,
                  const void* dL, void* dA, int32_t* info_dev, void* ws, size_t ws_bytes,
                  void* stream) {
  (void)batch; (void)opts; (void)A; (void)ctx; (void)dL; (void)dA; (void)info_dev;
  (void)ws; (void)ws_bytes; (void)stream;
  return LOGM_ERR_UNSUPPORTED;
}

}  // extern "C"
