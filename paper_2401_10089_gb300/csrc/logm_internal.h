// logm_internal.h -- host-side interface between the C ABI (logm_api.cu) and
// the kernel launchers. Not installed; the public surface is include/logm.h.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lg {

// Theta_{m_k} of the paper's backward-error table (Sec. 5), k = 1..6: the
// default bounds of the loop test and the order search (each entry point's
// options may override the first five; k = 6 is taken by the
// one-block-per-matrix kernels only).
constexpr double kThetaPaper[6] = {1.83e-8, 1.53e-4, 1.33e-2, 9.31e-2, 2.46e-1, 3.72e-1};

// Host set-up done once per device (e.g. a kernel's shared-memory attribute),
// safe when several threads drive several devices: run() calls f() with the
// caller's device current unless it already succeeded on that device
// (devices 64 and up: every time).
struct DeviceOnce {
  std::atomic<unsigned long long> done{0};
  template <class F>
  cudaError_t run(F f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = f();
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
  }
};

// Multiprocessor count of the current device (cached per device, thread safe).
int device_sm_count();

enum Mode : int { kModeExecute = 0, kModePlan = 1, kModeSqrt = 2, kModeGraph = 3, kModeBackward = 4 };

// Everything one launch of the one-block-per-matrix kernel needs. Device
// pointers unless noted.
struct SmallParams {
  // batch
  int count, dtype, n_uniform, n_max;
  int batch_nmax;  // n_max of the whole batch (n_max may be a configuration's smaller limit)
  const int32_t* n_dev;
  const int64_t* off_dev;
  // options
  int k_max, max_sqrt, max_db;
  int db_form;         // 0: eq. (ScalDB), two inversions per step; 1: product form
  int balance;         // 1: T^{-1} A T before and T L T^{-1} after (execute; backward reverses it)
  double* bal;         // balance: diag(T) per matrix, stride bal_stride (execute writes, backward reads)
  int bal_stride;      // the batch's n_max
  double theta[5];     // Theta_{m_k}, k = 1..5 (k = 4 unused)
  // inputs / outputs (NULL when unused by the mode)
  const void* A;       // execute, plan, sqrt (sqrt: in/out)
  void* A_inout;       // sqrt
  void* L;             // execute: L; graph: Z
  const void* AI2_in;  // plan
  void* A2_out;        // sqrt
  void* AI2_out;       // sqrt
  const void* X;       // graph
  const void* P3;      // graph
  const int32_t* k_in; // graph
  const int32_t* active;
  int32_t* s_out;
  int32_t* k_out;
  int32_t* info;
  int32_t* finish;
  double* alpha;
  int32_t* iters;
  int32_t* stats;      // execute: [4 * count] DB iterations, inverses, products, matvecs
  double* ctx;         // execute: per-level checkpoints (NULL = none); backward: read
  int32_t* ctx_hdr;    // execute: (s, k) per matrix for the backward (NULL = none)
  const void* dL;      // backward: adjoint of L
  void* dA;            // backward: result
  int ctx_levels;
  int ctx_nmax;        // n stride of the checkpoint layout (the batch's n_max)
  // workspace
  double* slots;       // n_slots * kSlotMats * n_max^2 doubles
  int32_t* queue;      // one counter, zeroed before the launch
  int32_t* order;      // execute: [count] queue position -> matrix, most expensive first (NULL: index order)
  int32_t* order_aux;  // [2 * kOrderBuckets + count]: bucket counts, bucket cursors, bucket per matrix
  int n_slots;
  int precision;       // graph products (FP64 in this kernel family)
  int fp64_tc;         // whole-GPU kernel: 1 = Gauss-Jordan updates on the tensor cores (exact BF16 digits)
  int large_pass;      // 1: matrices with n > kSmallMaxN are left to the whole-GPU kernel
  int bucket_mask;     // nonzero: only matrices whose size bucket bit is set (see size_bucket)
  float* gbuf;         // precision form: hand P_2, P_3 over in FP32 here and stop before the graph
  int gbuf_nmax;       // n stride of gbuf
};

// Parameters of the tensor-core graph stage (graph_tc.cu).
struct GraphParams {
  int count, n_uniform, n_max;
  const int32_t* n_dev;
  const int64_t* off_dev;
  const int32_t* k_dev;     // products per matrix (1..5)
  const int32_t* s_dev;     // square roots per matrix (scale -2^s), NULL: scale 1
  const int32_t* info_dev;  // matrices with info 1 or 4 are skipped; may be NULL
  float* gbuf;              // per matrix 5 slots of n_max^2 floats: P_2 .. P_6
  void* L;                  // output (dtype out_dtype) at the batch's offsets
  int out_dtype;
  int precision;            // LOGM_PREC_TF32X3 or LOGM_PREC_BF16X3
  int j;                    // product of this launch (1: P_3 = X X, 2..5)
  int p3_given;             // 1: slot 1 already holds P_3
  int32_t* err;             // set when a tensor-core wait timed out
  const double* bal;        // NULL, or diag(T) of the balancing per matrix (stride n_max): L <- T L T^{-1}
  void* pack;               // uniform batches: packed operand slices (graph_pack_bytes), else NULL
};

size_t graph_tc_smem_bytes();
cudaError_t launch_graph_tc(const GraphParams& p, cudaStream_t st);
cudaError_t launch_graph_k1(const GraphParams& p, cudaStream_t st);
// Uniform batches: pack + TMA-fed tcgen05 products (graph_tma.cu).
size_t graph_pack_bytes(int count, int n);
cudaError_t launch_graph_tma(const GraphParams& p, cudaStream_t st);
cudaError_t launch_graph_prep(const GraphParams& p, const void* X, const void* P3, int in_dtype, cudaStream_t st);

constexpr int kSlotMats = 7;
constexpr int kBwdTapeCap = 16;                       // Denman-Beavers iterations a backward level can reverse
constexpr int kBwdSlotMats = 7 + 6 + 4 + 2 * kBwdTapeCap;  // forward recompute, adjoints, temporaries, tape
size_t small_bwd_workspace_bytes(int count, int n_max);
constexpr int kOrderBuckets = 256;
constexpr int kCtxLevels = 12;
constexpr int kSmallMaxN = 256;  // largest n of the one-block-per-matrix kernels

int small_kernel_slots(int count);

// Size buckets of the one-block-per-matrix kernels: n <= 8, 16, 32, 64, 128, 256.
constexpr int kBuckets = 6;
constexpr int kBucketMaxN[kBuckets] = {8, 16, 32, 64, 128, 256};
__host__ __device__ inline int size_bucket(int n) {
  return n <= 8 ? 0 : (n <= 16 ? 1 : (n <= 32 ? 2 : (n <= 64 ? 3 : (n <= 128 ? 4 : 5))));
}
size_t large_workspace_bytes(int n_max);
cudaError_t launch_large(Mode mode, const SmallParams& p, void* ws, cudaStream_t stream);
cudaError_t launch_barrier_probe(int missing, unsigned long long timeout_ns, void* ws, cudaStream_t stream);
size_t small_workspace_bytes(int count, int n_max);
size_t small_order_bytes(int count);
cudaError_t launch_small(Mode mode, const SmallParams& p, cudaStream_t stream);

}  // namespace lg

// The other configurations of the one-block-per-matrix kernel (same sources,
// built in their own translation units): lg_v1 = 128 threads, n <= 64,
// 32 x 32 DMMA tiles; lg_v2 = 64 threads, n <= 32, 32 x 32 tiles.
namespace lg_v1 {
constexpr int kVariantMaxN = 64;
int small_kernel_slots(int count);
size_t small_bwd_workspace_bytes(int count, int n_max);
size_t small_workspace_bytes(int count, int n_max);
cudaError_t launch_small(lg::Mode mode, const lg::SmallParams& p, cudaStream_t stream);
}  // namespace lg_v1
namespace lg_v2 {
constexpr int kVariantMaxN = 32;
int small_kernel_slots(int count);
size_t small_bwd_workspace_bytes(int count, int n_max);
size_t small_workspace_bytes(int count, int n_max);
cudaError_t launch_small(lg::Mode mode, const lg::SmallParams& p, cudaStream_t stream);
}  // namespace lg_v2
namespace lg_v3 {
constexpr int kVariantMaxN = 256;
int small_kernel_slots(int count);
size_t small_bwd_workspace_bytes(int count, int n_max);
size_t small_workspace_bytes(int count, int n_max);
cudaError_t launch_small(lg::Mode mode, const lg::SmallParams& p, cudaStream_t stream);
}  // namespace lg_v3
// lg_v5 = lg_v2 with the execute mode's working matrices in shared memory.
namespace lg_v5 {
constexpr int kVariantMaxN = 32;
int small_kernel_slots(int count);
size_t small_bwd_workspace_bytes(int count, int n_max);
size_t small_workspace_bytes(int count, int n_max);
cudaError_t launch_small(lg::Mode mode, const lg::SmallParams& p, cudaStream_t stream);
}  // namespace lg_v5
// lg_v4 = lg_v1 with seven blocks per SM (one round for uniform batches of
// 5..7 matrices per SM).
namespace lg_v4 {
constexpr int kVariantMaxN = 64;
int small_kernel_slots(int count);
size_t small_bwd_workspace_bytes(int count, int n_max);
size_t small_workspace_bytes(int count, int n_max);
cudaError_t launch_small(lg::Mode mode, const lg::SmallParams& p, cudaStream_t stream);
}  // namespace lg_v4
