// logm_api.cu -- the extern "C" entry points declared in include/logm.h.
// Argument checking, workspace layout and dispatch; every step of the method
// runs in the kernels this file launches.
#include <cstdint>
#include <cstring>

#include "../../include/logm.h"
#include "logm_internal.h"

namespace lg {

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  const bool cached = dev >= 0 && dev < 64;
  if (cached) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1;
  if (cached) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

}  // namespace lg

namespace {

// Kernel configuration per size bucket (logm_set_tuning).
int g_variant[lg::kBuckets] = {0, 0, 0, 0, 0, 0};
constexpr int kVariants = 5;  // tunable configurations; configuration 1's 7-per-SM twin is picked by batch size
constexpr int kVariantMaxBucket[kVariants] = {5, 3, 2, 5, 2};  // largest bucket each configuration serves

size_t small_slots_bytes_all_variants(int count, int small_nmax) {
  size_t m = lg::small_workspace_bytes(count, small_nmax);
  const size_t m1 = lg_v1::small_workspace_bytes(count, small_nmax < 64 ? small_nmax : 64);
  const size_t m2 = lg_v2::small_workspace_bytes(count, small_nmax < 32 ? small_nmax : 32);
  const size_t m3 = lg_v3::small_workspace_bytes(count, small_nmax);
  const size_t m4 = lg_v4::small_workspace_bytes(count, small_nmax < 64 ? small_nmax : 64);
  const size_t m5 = lg_v5::small_workspace_bytes(count, small_nmax < 32 ? small_nmax : 32);
  if (m5 > m) m = m5;
  if (m4 > m) m = m4;
  if (m1 > m) m = m1;
  if (m2 > m) m = m2;
  if (m3 > m) m = m3;
  return m;
}

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
  if (o->k_max < 1 || o->k_max > 6) return 0;
  if (o->precision < LOGM_PREC_FP64 || o->precision > LOGM_PREC_BF16X3) return 0;
  if (o->k_max == 6 && o->precision != LOGM_PREC_FP64) return 0;  // split-precision graph: k <= 5
  if (o->max_sqrt < 0 || o->max_sqrt > 1000) return 0;
  if (o->max_db_iter < 1 || o->max_db_iter > 1000) return 0;
  if (o->db_form != LOGM_DB_TWO_INVERSE && o->db_form != LOGM_DB_PRODUCT) return 0;
  if (o->balance != LOGM_BALANCE_NONE && o->balance != LOGM_BALANCE_SCALE) return 0;
  if (o->fp64_products != LOGM_FP64_PIPE && o->fp64_products != LOGM_FP64_TC_SLICED) return 0;
  for (int t = 0; t < 5; ++t)
    if (!(o->theta[t] >= 0.0) || !(o->theta[t] < 1.0)) return 0;
  return 1;
}

// Workspace: [small part | large part]. The small part (queue, order, one
// slot of kSlotMats matrices per resident block) serves matrices with
// n <= kSmallMaxN; the large part (one whole-GPU slot) serves n > kSmallMaxN.
struct WsLayout {
  int small_nmax;   // 0: no small pass
  int large_nmax;   // 0: no large pass
  size_t small_bytes, large_off, bal_off, graph_off, total;
};

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Tensor-core graph stage region: FP32 slots P_2 .. P_6 per matrix, then k, s
// (when the caller passes none), an error word and, for uniform batches, the
// packed operand slices of the TMA-fed product kernel.
size_t graph_region_bytes(const logm_batch* b, int n_max) {
  return round256(sizeof(float) * 5 * (size_t)b->count * n_max * n_max) +
         2 * round256(sizeof(int32_t) * (size_t)b->count) + 256 +
         (b->n_uniform > 0 ? round256(lg::graph_pack_bytes(b->count, n_max)) : 0);
}

WsLayout ws_layout(const logm_batch* b, int precision) {
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
  L.small_bytes = L.small_nmax ? small_slots_bytes_all_variants(b->count, L.small_nmax) : 0;
  L.large_off = round256(L.small_bytes);
  // diag(T) of the balancing, per matrix (used when no context is given)
  L.bal_off = round256(L.large_off + (L.large_nmax ? lg::large_workspace_bytes(L.large_nmax) : 0));
  L.graph_off = round256(L.bal_off + sizeof(double) * (size_t)b->count * n_max);
  L.total = L.graph_off + (precision != LOGM_PREC_FP64 ? graph_region_bytes(b, n_max) : 0);
  return L;
}

struct GraphRegion {
  float* gbuf;
  int32_t* k;
  int32_t* s;
  int32_t* err;
  void* pack;  // uniform batches only
};

GraphRegion graph_region(const logm_batch* b, const WsLayout& L, void* ws) {
  char* w = static_cast<char*>(ws) + L.graph_off;
  const int n_max = batch_n_max(b);
  GraphRegion g;
  g.gbuf = reinterpret_cast<float*>(w);
  w += round256(sizeof(float) * 5 * (size_t)b->count * n_max * n_max);
  g.k = reinterpret_cast<int32_t*>(w);
  w += round256(sizeof(int32_t) * (size_t)b->count);
  g.s = reinterpret_cast<int32_t*>(w);
  w += round256(sizeof(int32_t) * (size_t)b->count);
  g.err = reinterpret_cast<int32_t*>(w);
  w += 256;
  g.pack = b->n_uniform > 0 ? static_cast<void*>(w) : nullptr;
  return g;
}

void fill_common(lg::SmallParams& p, const logm_batch* b, const logm_options* o) {
  std::memset(&p, 0, sizeof(p));
  p.count = b->count;
  p.dtype = b->dtype;
  p.n_uniform = b->n_uniform > 0 ? b->n_uniform : 0;
  p.n_max = batch_n_max(b);
  p.batch_nmax = p.n_max;
  p.n_dev = b->n;
  p.off_dev = b->offset;
  if (o) {
    p.k_max = o->k_max;
    p.max_sqrt = o->max_sqrt;
    p.max_db = o->max_db_iter;
    for (int t = 0; t < 5; ++t) p.theta[t] = o->theta[t] > 0.0 ? o->theta[t] : lg::kThetaPaper[t];
    p.precision = o->precision;
    p.db_form = o->db_form;
    p.balance = o->balance;
    p.fp64_tc = o->fp64_products == LOGM_FP64_TC_SLICED;
  } else {
    p.k_max = 5;
    p.max_sqrt = 40;
    p.max_db = 50;
    for (int t = 0; t < 5; ++t) p.theta[t] = lg::kThetaPaper[t];
  }
  p.ctx_nmax = p.n_max;
  p.bal_stride = p.n_max;
}

// One launch per block configuration, each taking the size buckets the
// tuning table gives it (execute and backward; the other entry points use
// configuration 0 for every bucket).
cudaError_t launch_small_variants(lg::Mode mode, const lg::SmallParams& q, int small_nmax, int count,
                                  cudaStream_t st) {
  const bool tuned = mode == lg::kModeExecute || mode == lg::kModeBackward;
  int mask[kVariants] = {0, 0, 0, 0, 0};
  const int top = lg::size_bucket(small_nmax);
  // a uniform batch fills one bucket: only its configuration is launched
  const int lo = q.n_uniform > 0 ? top : 0;
  for (int bk = lo; bk <= top; ++bk) mask[tuned ? g_variant[bk] : 0] |= 1 << bk;
  if (lo == 0 && mask[0] == (1 << (top + 1)) - 1) mask[0] = 0;  // configuration 0 takes everything: no filter
  if (lo > 0 && mask[0]) mask[0] = 0;  // configuration 0 holds the only bucket: no filter
  for (int v = kVariants - 1; v >= 0; --v) {
    if (v > 0 && !mask[v]) continue;
    if (v == 0 && !mask[0] && (mask[1] || mask[2] || mask[3] || mask[4])) continue;
    lg::SmallParams r = q;
    r.bucket_mask = mask[v];
    cudaError_t e;
    if (v == 0) {
      r.n_slots = lg::small_kernel_slots(count);
      e = lg::launch_small(mode, r, st);
    } else if (v == 1) {
      r.n_max = q.n_max < 64 ? q.n_max : 64;
      const int s1 = lg_v1::small_kernel_slots(count), s4 = lg_v4::small_kernel_slots(count);
      if (q.n_uniform > 0 && count > s1 && count <= s4) {  // one round at 7 per SM instead of two at 5
        r.n_slots = s4;
        e = lg_v4::launch_small(mode, r, st);
      } else {
        r.n_slots = s1;
        e = lg_v1::launch_small(mode, r, st);
      }
    } else if (v == 2) {
      r.n_max = q.n_max < 32 ? q.n_max : 32;
      r.n_slots = lg_v2::small_kernel_slots(count);
      e = lg_v2::launch_small(mode, r, st);
    } else if (v == 4) {
      r.n_max = q.n_max < 32 ? q.n_max : 32;
      r.n_slots = lg_v5::small_kernel_slots(count);  // execute sizes its grid by occupancy
      e = lg_v5::launch_small(mode, r, st);
    } else {
      r.n_slots = lg_v3::small_kernel_slots(count);
      e = lg_v3::launch_small(mode, r, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Launch the small pass and/or the large pass for this batch.
int run_passes(lg::Mode mode, lg::SmallParams& p, const logm_batch* b, void* ws, cudaStream_t st) {
  const WsLayout L = ws_layout(b, LOGM_PREC_FP64);
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
    if (launch_small_variants(mode, q, L.small_nmax, b->count, st) != cudaSuccess) return LOGM_ERR_CUDA;
  }
  if (L.large_nmax) {
    lg::SmallParams q = p;
    q.n_max = L.large_nmax;
    q.large_pass = L.small_nmax ? 1 : 0;
    if (lg::launch_large(mode, q, w + L.large_off, st) != cudaSuccess) return LOGM_ERR_CUDA;
  }
  return LOGM_SUCCESS;
}

// Split-precision graph products: uniform batches take the packed TMA-fed
// kernels (graph_tma.cu), ragged ones the kernel that forms its operand
// tiles in shared memory (graph_tc.cu); k = 1 matrices need no product.
cudaError_t launch_graph_products(const lg::GraphParams& gp, cudaStream_t st) {
  if (gp.pack) {
    cudaError_t e = lg::launch_graph_tma(gp, st);
    if (e != cudaSuccess) return e;
    return lg::launch_graph_k1(gp, st);
  }
  return lg::launch_graph_tc(gp, st);
}

int check_ws(const logm_batch* b, void* ws, size_t ws_bytes, int precision = LOGM_PREC_FP64) {
  if (!ws) return LOGM_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return LOGM_ERR_WORKSPACE;
  if (ws_bytes < ws_layout(b, precision).total) return LOGM_ERR_WORKSPACE;
  return LOGM_SUCCESS;
}

}  // namespace

extern "C" {

int logm_version(void) { return 200; }

// Host-buffer entry: [logm_execute workspace | A copy | L copy | s | k | info].
// The inner workspace comes first, at the caller's (allocation-aligned) base:
// placed after the two copies it measured up to 5 % slower.
static size_t host_matrix_bytes(const logm_batch* b) {
  const size_t esz = b->dtype == LOGM_DTYPE_F64 ? 8 : 4;
  return (size_t)b->count * (size_t)b->n_uniform * (size_t)b->n_uniform * esz;
}

size_t logm_host_workspace_size(const logm_batch* batch, const logm_options* opts) {
  if (!batch || batch->n_uniform <= 0 || batch_n_max(batch) <= 0) return 0;
  const size_t inner = logm_workspace_size(batch, opts);
  if (inner == 0) return 0;
  return round256(inner) + 2 * round256(host_matrix_bytes(batch)) + round256(3 * sizeof(int32_t) * (size_t)batch->count);
}

int logm_execute_host(const logm_batch* batch, const logm_options* opts, const void* A_host, void* L_host,
                      int32_t* s_host, int32_t* k_host, int32_t* info_host, void* ws, size_t ws_bytes,
                      void* stream) {
  if (batch_n_max(batch) <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (batch->n_uniform <= 0) return LOGM_ERR_UNSUPPORTED;
  if (opts->k_max == 6 && batch->n_uniform > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A_host || !L_host || !info_host) return LOGM_ERR_INVALID_ARG;
  const size_t need = logm_host_workspace_size(batch, opts);
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < need) return LOGM_ERR_WORKSPACE;
  const size_t mb = host_matrix_bytes(batch), mr = round256(mb);
  const size_t cnt = (size_t)batch->count;
  const size_t inner_bytes = round256(logm_workspace_size(batch, opts));
  char* inner = static_cast<char*>(ws);
  char* w = inner + inner_bytes;
  void* A_dev = w;
  void* L_dev = w + mr;
  int32_t* s_dev = reinterpret_cast<int32_t*>(w + 2 * mr);
  int32_t* k_dev = s_dev + cnt;
  int32_t* info_dev = k_dev + cnt;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(A_dev, A_host, mb, cudaMemcpyHostToDevice, st) != cudaSuccess) return LOGM_ERR_CUDA;
  const int r = logm_execute(batch, opts, A_dev, L_dev, s_dev, k_dev, info_dev, nullptr, nullptr, inner,
                             inner_bytes, stream);
  if (r != LOGM_SUCCESS) return r;
  if (cudaMemcpyAsync(L_host, L_dev, mb, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LOGM_ERR_CUDA;
  const size_t ib = sizeof(int32_t) * cnt;
  if (s_host && cudaMemcpyAsync(s_host, s_dev, ib, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LOGM_ERR_CUDA;
  if (k_host && cudaMemcpyAsync(k_host, k_dev, ib, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LOGM_ERR_CUDA;
  if (cudaMemcpyAsync(info_host, info_dev, ib, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LOGM_ERR_CUDA;
  return LOGM_SUCCESS;
}

int logm_probe_barrier(int32_t missing, double timeout_s, void* ws, size_t ws_bytes, void* stream) {
  if (missing < 0 || missing > 8 || !(timeout_s >= 1e-6 && timeout_s <= 60.0)) return LOGM_ERR_INVALID_ARG;
  if (!ws || ws_bytes < 16 || reinterpret_cast<uintptr_t>(ws) % 8 != 0) return LOGM_ERR_WORKSPACE;
  const unsigned long long ns = static_cast<unsigned long long>(timeout_s * 1e9);
  if (lg::launch_barrier_probe(missing, ns, ws, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LOGM_ERR_CUDA;
  return LOGM_SUCCESS;
}

int logm_set_tuning(const logm_tuning* t) {
  if (!t) {
    for (int b = 0; b < lg::kBuckets; ++b) g_variant[b] = 0;
    return LOGM_SUCCESS;
  }
  for (int b = 0; b < lg::kBuckets; ++b) {
    const int v = t->variant[b];
    if (v < 0 || v >= kVariants || b > kVariantMaxBucket[v]) return LOGM_ERR_INVALID_ARG;
  }
  for (int b = 0; b < lg::kBuckets; ++b) g_variant[b] = t->variant[b];
  return LOGM_SUCCESS;
}

int logm_get_tuning(logm_tuning* t) {
  if (!t) return LOGM_ERR_INVALID_ARG;
  for (int b = 0; b < lg::kBuckets; ++b) t->variant[b] = g_variant[b];
  return LOGM_SUCCESS;
}

size_t logm_workspace_size(const logm_batch* batch, const logm_options* opts) {
  if (batch_n_max(batch) <= 0) return 0;
  return ws_layout(batch, opts ? opts->precision : LOGM_PREC_TF32X3).total;
}

// Context: (s, k) per matrix, diag(T) of the balancing per matrix, then the
// input of every square-root level.
size_t ctx_header_bytes(const logm_batch* b) { return round256(sizeof(int32_t) * 2 * (size_t)b->count); }
size_t ctx_bal_bytes(const logm_batch* b) {
  return round256(sizeof(double) * (size_t)b->count * (size_t)batch_n_max(b));
}

size_t logm_context_size(const logm_batch* batch, const logm_options* opts) {
  (void)opts;
  const int n_max = batch_n_max(batch);
  if (n_max <= 0) return 0;
  return ctx_header_bytes(batch) + ctx_bal_bytes(batch) +
         (size_t)batch->count * lg::kCtxLevels * (size_t)n_max * n_max * sizeof(double);
}

size_t logm_backward_workspace_size(const logm_batch* batch, const logm_options* opts) {
  (void)opts;
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || n_max > lg::kSmallMaxN) return 0;
  size_t m = lg::small_bwd_workspace_bytes(batch->count, n_max);
  const size_t m1 = lg_v1::small_bwd_workspace_bytes(batch->count, n_max < 64 ? n_max : 64);
  const size_t m2 = lg_v2::small_bwd_workspace_bytes(batch->count, n_max < 32 ? n_max : 32);
  const size_t m3 = lg_v3::small_bwd_workspace_bytes(batch->count, n_max);
  const size_t m4 = lg_v4::small_bwd_workspace_bytes(batch->count, n_max < 64 ? n_max : 64);
  const size_t m5 = lg_v5::small_bwd_workspace_bytes(batch->count, n_max < 32 ? n_max : 32);
  size_t r = m > m1 ? m : m1;
  r = r > m4 ? r : m4;
  r = r > m5 ? r : m5;
  r = r > m2 ? r : m2;
  return r > m3 ? r : m3;
}

int logm_plan(const logm_batch* batch, const logm_options* opts, const void* A, const void* AI2,
              int32_t* finish_dev, int32_t* k_dev, double* alpha_dev, int32_t* info_dev, void* ws,
              size_t ws_bytes, void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (opts->k_max == 6 && n_max > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
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
  if (int r = check_ws(batch, ws, ws_bytes, precision)) return r;
  if (precision != LOGM_PREC_FP64) {
    const WsLayout L = ws_layout(batch, precision);
    const GraphRegion g = graph_region(batch, L, ws);
    lg::GraphParams gp{};
    gp.count = batch->count;
    gp.n_uniform = batch->n_uniform > 0 ? batch->n_uniform : 0;
    gp.n_max = n_max;
    gp.n_dev = batch->n;
    gp.off_dev = batch->offset;
    gp.k_dev = k_dev;
    gp.s_dev = nullptr;
    gp.info_dev = nullptr;
    gp.gbuf = g.gbuf;
    gp.L = Z;
    gp.out_dtype = batch->dtype;
    gp.precision = precision;
    gp.p3_given = P3 ? 1 : 0;
    gp.err = g.err;
    gp.pack = g.pack;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(g.err, 0, sizeof(int32_t), st) != cudaSuccess) return LOGM_ERR_CUDA;
    if (lg::launch_graph_prep(gp, X, P3, batch->dtype, st) != cudaSuccess) return LOGM_ERR_CUDA;
    return launch_graph_products(gp, st) == cudaSuccess ? LOGM_SUCCESS : LOGM_ERR_CUDA;
  }
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
  // k = 6: one-block-per-matrix kernels only, and no adjoint for it
  if (opts->k_max == 6 && (n_max > lg::kSmallMaxN || ctx)) return LOGM_ERR_UNSUPPORTED;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !L || !info_dev) return LOGM_ERR_INVALID_ARG;
  if (int r = check_ws(batch, ws, ws_bytes, opts->precision)) return r;
  lg::SmallParams p;
  fill_common(p, batch, opts);
  p.A = A;
  p.L = L;
  p.s_out = s_dev;
  p.k_out = k_dev;
  p.info = info_dev;
  p.stats = stats_dev;
  if (ctx) {
    p.ctx_hdr = static_cast<int32_t*>(ctx);
    p.bal = reinterpret_cast<double*>(static_cast<char*>(ctx) + ctx_header_bytes(batch));
    p.ctx = reinterpret_cast<double*>(static_cast<char*>(ctx) + ctx_header_bytes(batch) + ctx_bal_bytes(batch));
  } else {
    p.bal = reinterpret_cast<double*>(static_cast<char*>(ws) + ws_layout(batch, opts->precision).bal_off);
  }
  p.ctx_levels = lg::kCtxLevels;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (opts->precision == LOGM_PREC_FP64) return run_passes(lg::kModeExecute, p, batch, ws, st);
  // precision form: FP64 plan and square roots, then the graph products on the tensor cores
  const WsLayout L2 = ws_layout(batch, opts->precision);
  const GraphRegion g = graph_region(batch, L2, ws);
  p.gbuf = g.gbuf;
  p.gbuf_nmax = n_max;
  if (!p.k_out) p.k_out = g.k;
  if (!p.s_out) p.s_out = g.s;
  if (int r = run_passes(lg::kModeExecute, p, batch, ws, st)) return r;
  lg::GraphParams gp{};
  gp.count = batch->count;
  gp.n_uniform = batch->n_uniform > 0 ? batch->n_uniform : 0;
  gp.n_max = n_max;
  gp.n_dev = batch->n;
  gp.off_dev = batch->offset;
  gp.k_dev = p.k_out;
  gp.s_dev = p.s_out;
  gp.info_dev = info_dev;
  gp.gbuf = g.gbuf;
  gp.L = L;
  gp.out_dtype = batch->dtype;
  gp.precision = opts->precision;
  gp.p3_given = 1;
  gp.err = g.err;
  gp.bal = p.balance ? p.bal : nullptr;
  gp.pack = g.pack;
  if (cudaMemsetAsync(g.err, 0, sizeof(int32_t), st) != cudaSuccess) return LOGM_ERR_CUDA;
  return launch_graph_products(gp, st) == cudaSuccess ? LOGM_SUCCESS : LOGM_ERR_CUDA;
}

int logm_backward(const logm_batch* batch, const logm_options* opts, const void* A, const void* ctx,
                  const void* dL, void* dA, int32_t* info_dev, void* ws, size_t ws_bytes,
                  void* stream) {
  const int n_max = batch_n_max(batch);
  if (n_max <= 0 || !opts_ok(opts)) return LOGM_ERR_INVALID_ARG;
  if (opts->k_max == 6) return LOGM_ERR_UNSUPPORTED;
  if (batch->count == 0) return LOGM_SUCCESS;
  if (!A || !ctx || !dL || !dA || !info_dev) return LOGM_ERR_INVALID_ARG;
  if (n_max > lg::kSmallMaxN) return LOGM_ERR_UNSUPPORTED;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return LOGM_ERR_WORKSPACE;
  if (ws_bytes < logm_backward_workspace_size(batch, opts)) return LOGM_ERR_WORKSPACE;
  lg::SmallParams p;
  fill_common(p, batch, opts);
  p.A = A;
  p.dL = dL;
  p.dA = dA;
  p.info = info_dev;
  p.ctx_hdr = const_cast<int32_t*>(static_cast<const int32_t*>(ctx));
  char* cb = const_cast<char*>(static_cast<const char*>(ctx));
  p.bal = reinterpret_cast<double*>(cb + ctx_header_bytes(batch));
  p.ctx = reinterpret_cast<double*>(cb + ctx_header_bytes(batch) + ctx_bal_bytes(batch));
  p.ctx_levels = lg::kCtxLevels;
  char* w = static_cast<char*>(ws);
  p.queue = reinterpret_cast<int32_t*>(w);
  p.slots = reinterpret_cast<double*>(w + 256 + lg::small_order_bytes(batch->count));
  const cudaError_t e =
      launch_small_variants(lg::kModeBackward, p, n_max, batch->count, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LOGM_SUCCESS : LOGM_ERR_CUDA;
}

}  // extern "C"
