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

void fill_common(lg::SmallParams& p, const logm_batch* b, const logm_options* o, void* ws) {
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
  char* w = static_cast<char*>(ws);
  p.queue = reinterpret_cast<int32_t*>(w);
  const size_t ob = lg::small_order_bytes(b->count);
  p.order = reinterpret_cast<int32_t*>(w + 256);
  p.order_aux = p.order + b->count;
  p.slots = reinterpret_cast<double*>(w + 256 + ob);
  p.n_slots = lg::small_kernel_slots(b->count);
}

int check_ws(const logm_batch* b, const logm_options* o, void* ws, size_t ws_bytes) {
  if (!ws) return LOGM_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return LOGM_ERR_WORKSPACE;
  if (ws_bytes < logm_workspace_size(b, o)) return LOGM_ERR_WORKSPACE;
  return LOGM_SUCCESS;
}

int finish_launch(cudaError_t e) { return e == cudaSuccess ? LOGM_SUCCESS : LOGM_ERR_CUDA; }

}  // namespace

extern "C" {

int logm_version(void) { return 100; }

size_t logm_workspace_size(const logm_batch* batch, const logm_options* opts) {
  (void)opts;
  const int n_max = batch_n_max(batch);
  if (n_max <= 0) return 0;
  if (n_max > lg::kSmallMaxN) return 0;
  return lg::small_workspace_bytes(batch->count, n_max);
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
  if (n_max > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
  if (int r = check_ws(batch, opts, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, opts, ws);
  p.A = A;
  p.AI2_in = AI2;
  p.finish = finish_dev;
  p.k_out = k_dev;
  p.alpha = alpha_dev;
  p.info = info_dev;
  return finish_launch(lg::launch_small(lg::kModePlan, p, static_cast<cudaStream_t>(stream)));
}

int logm_sqrt(const logm_batch* batch, const logm_options* opts, void* A, void* A2_out,
              void* AI2_out, const int32_t* active_dev, int32_t* iters_dev, int32_t* info_dev,
              void* ws, size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !info_dev) return LOGM_ERR_INVALID_ARG;
  if (n_max > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
  if (int r = check_ws(batch, opts, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, opts, ws);
  p.A_inout = A;
  p.A2_out = A2_out;
  p.AI2_out = AI2_out;
  p.active = active_dev;
  p.iters = iters_dev;
  p.info = info_dev;
  return finish_launch(lg::launch_small(lg::kModeSqrt, p, static_cast<cudaStream_t>(stream)));
}

int logm_graph_eval(const logm_batch* batch, int32_t precision, const void* X, const void* P3,
                    const int32_t* k_dev, void* Z, void* ws, size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0) return LOGM_ERR_INVALID_ARG;
  if (precision < LOGM_PREC_FP64 || precision > LOGM_PREC_BF16X3) return LOGM_ERR_INVALID_ARG;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!X || !k_dev || !Z) return LOGM_ERR_INVALID_ARG;
  if (n_max > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
  if (precision != LOGM_PREC_FP64) return LOGM_ERR_UNSUPPORTED;
  if (int r = check_ws(batch, nullptr, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, nullptr, ws);
  p.X = X;
  p.P3 = P3;
  p.k_in = k_dev;
  p.L = Z;
  p.precision = precision;
  return finish_launch(lg::launch_small(lg::kModeGraph, p, static_cast<cudaStream_t>(stream)));
}

int logm_execute(const logm_batch* batch, const logm_options* opts, const void* A, void* L,
                 int32_t* s_dev, int32_t* k_dev, int32_t* info_dev, int32_t* stats_dev, void* ctx,
                 void* ws, size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !L || !info_dev) return LOGM_ERR_INVALID_ARG;
  if (n_max > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
  if (opts->precision != LOGM_PREC_FP64) return LOGM_ERR_UNSUPPORTED;
  if (int r = check_ws(batch, opts, ws, ws_bytes)) return r;
  lg::SmallParams p;
  fill_common(p, batch, opts, ws);
  p.A = A;
  p.L = L;
  p.s_out = s_dev;
  p.k_out = k_dev;
  p.info = info_dev;
  p.stats = stats_dev;
  p.ctx = static_cast<double*>(ctx);
  p.ctx_levels = lg::kCtxLevels;
  return finish_launch(lg::launch_small(lg::kModeExecute, p, static_cast<cudaStream_t>(stream)));
}

int logm_backward(const logm_batch* batch, const logm_options* opts, const void* A, const void* ctx,
                  const void* dL, void* dA, int32_t* info_dev, void* ws, size_t ws_bytes,
                  void* stream) {
  (void)batch; (void)opts; (void)A; (void)ctx; (void)dL; (void)dA; (void)info_dev;
  (void)ws; (void)ws_bytes; (void)stream;
  return LOGM_ERR_UNSUPPORTED;
}

}  // extern "C"
