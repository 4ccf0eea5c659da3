// logm_small.cu -- Algorithm 1 of arXiv 2401.10089 (Sec. 6) with one thread
// block per matrix, for n <= kMaxN. A persistent grid pulls matrices from a
// device work queue, so a ragged batch of thousands of matrices is one launch
// and every data-dependent loop (square-root count s, Denman-Beavers
// iterations, estimator sweeps) runs on the device with no host round trip.
//
// Per block, the working matrices live in a workspace slot of kSlotMats
// n_max x n_max FP64 buffers (L2-resident; with LG_SMEM_SLOTS the execute
// mode keeps them in the block's shared memory instead):
//   Acur  current A (the Denman-Beavers X in place), later P_2 = X = I - A
//   A2    saved A_2, then A_I2 = A_2 - 2A + I (eq. AI2) = P_3
//   Y     Denman-Beavers Y, later P_4
//   W1,W2 inverses of X and Y, later P_5, P_6
//   T1,T2 lin-comb nodes (the two factors of the next product)
// These kernels also take k = 6 (the graph of logm_algo.cuh fits it in the
// same seven matrices).
#include <cmath>
#include <cstdio>

#define LG_WITH_K6 1
#include "logm_internal.h"
#include "block_ops.cuh"
#include "logm_algo.cuh"

#ifndef LG_SMEM_SLOTS
#define LG_SMEM_SLOTS 0
#endif

namespace LG_NS {

// Byte offset of the shared-memory slot after the block's BlockSmem.
constexpr size_t kSmemSlotOffset = (sizeof(BlockSmem) + 255) / 256 * 256;
// Shared-memory slot mode: execute keeps its slot in shared memory.
template <int MODE>
__host__ __device__ constexpr bool smem_slot() {
  return LG_SMEM_SLOTS && MODE == kModeExecute;
}

// ---------------------------------------------------------------------------
// Queue order for execute: longest work first. The cost of a matrix grows
// with n^3 and with the number of square roots, which grows with
// log(||A - I||_1 / Theta); a counting sort over log-scale buckets of
// n^3 (1 + log2(1 + ||A - I||_1 / Theta)) puts the expensive matrices at the
// head of the queue so the tail of the persistent grid holds only cheap ones.
// Scheduling only: every matrix's arithmetic is the same in any order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_order_keys(SmallParams p) {
  __shared__ Reduce red;
  int* hist = p.order_aux;
  int* bucket_of = p.order_aux + 2 * kOrderBuckets;
  const double th = LG_THETA(p.theta, p.k_max);
  for (int b = blockIdx.x; b < p.count; b += gridDim.x) {
    int n;
    int64_t off;
    matrix_geometry(p, b, &n, &off);
    double best = 0.0;
    // matrices another configuration (or the whole-GPU kernel) takes are not
    // read: they go to the cheapest bucket, at the end of this queue
    const bool mine = !(p.bucket_mask && !((p.bucket_mask >> size_bucket(n)) & 1)) && !(n > kMaxN && p.large_pass);
    if (mine && n >= 1 && n <= p.n_max) {
      for (int j = threadIdx.x; j < n; j += kThreads) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) {
          double v = load_elem(p.A, p.dtype, off + (int64_t)i * n + j);
          if (i == j) v -= 1.0;
          sum += fabs(v);
        }
        best = nanmax(best, sum);
      }
    }
    const double nu = block_max(best, red);
    if (threadIdx.x == 0) {
      const double n3 = (mine && n >= 1 ? (double)n * n * n : 0.0);
      double key = n3 * (1.0 + log2(1.0 + (nu == nu ? nu : 1e30) / th));
      int bk = (int)(4.0 * log2(key + 1.0));
      bk = bk < 0 ? 0 : (bk >= kOrderBuckets ? kOrderBuckets - 1 : bk);
      bucket_of[b] = bk;
      atomicAdd(&hist[bk], 1);
    }
    __syncthreads();
  }
}

// Exclusive scan with the largest bucket first: cursor[bk] = first queue slot of bucket bk.
__global__ void k_order_scan(SmallParams p) {
  if (threadIdx.x == 0) {
    int* hist = p.order_aux;
    int* cursor = p.order_aux + kOrderBuckets;
    int acc = 0;
    for (int bk = kOrderBuckets - 1; bk >= 0; --bk) {
      cursor[bk] = acc;
      acc += hist[bk];
    }
  }
}

__global__ void k_order_scatter(SmallParams p) {
  int* cursor = p.order_aux + kOrderBuckets;
  const int* bucket_of = p.order_aux + 2 * kOrderBuckets;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < p.count; b += gridDim.x * blockDim.x) {
    const int pos = atomicAdd(&cursor[bucket_of[b]], 1);
    p.order[pos] = b;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, LG_MINBLOCKS) k_logm_small(SmallParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSmem& S = *reinterpret_cast<BlockSmem*>(smem_raw);
  BlockOps ops{S};
  const int64_t nn_max = (int64_t)p.n_max * p.n_max;
  const int mats = (MODE == kModeBackward) ? kBwdSlotMats : kSlotMats;
  double* base = smem_slot<MODE>() ? reinterpret_cast<double*>(smem_raw + kSmemSlotOffset)
                                   : p.slots + (int64_t)blockIdx.x * mats * nn_max;
  Slot M{base, base + nn_max, base + 2 * nn_max, base + 3 * nn_max,
         base + 4 * nn_max, base + 5 * nn_max, base + 6 * nn_max};
  BwdSlot W;
  if (MODE == kModeBackward) {
    W.F = M;
    for (int i = 0; i < 6; ++i) W.Pb[i] = base + (7 + i) * nn_max;
    W.Lb = base + 13 * nn_max;
    W.Rb = base + 14 * nn_max;
    W.Ab = base + 15 * nn_max;
    W.Yb = base + 16 * nn_max;
    W.tape.inv = base + 17 * nn_max;
    W.tape.stride = nn_max;
    W.tape.cap = kBwdTapeCap;
    W.tape.mu = p.slots + (int64_t)p.n_slots * kBwdSlotMats * nn_max + (int64_t)blockIdx.x * kBwdTapeCap;
  }
  for (;;) {
    if (threadIdx.x == 0) S.ibc[0] = atomicAdd(p.queue, 1);
    __syncthreads();
    const int q = S.ibc[0];
    __syncthreads();
    if (q >= p.count) break;
    const int b = p.order ? p.order[q] : q;
    int n;
    int64_t off;
    matrix_geometry(p, b, &n, &off);
    if (n < 1 || n > p.batch_nmax) {
      // a size no kernel may take: refused once, by the configuration that
      // owns the smallest bucket (the whole-GPU kernel refuses n > n_max when
      // it runs), and never read
      const bool owner = p.bucket_mask == 0 || (p.bucket_mask & 1);
      if (owner && !(n > kMaxN && p.large_pass) && threadIdx.x == 0) {
        if (p.info) p.info[b] = -1;
        if (p.s_out) p.s_out[b] = 0;
        if (p.k_out) p.k_out[b] = p.k_max;
      }
      continue;
    }
    if (p.bucket_mask && !((p.bucket_mask >> size_bucket(n)) & 1)) continue;  // another configuration's
    if (n > kMaxN && p.large_pass) continue;  // handled by the whole-GPU kernel
    if (n > kMaxN || n > p.n_max) {
      if (threadIdx.x == 0) {
        if (p.info) p.info[b] = -1;
        if (p.s_out) p.s_out[b] = 0;
        if (p.k_out) p.k_out[b] = p.k_max;
      }
      continue;
    }
    if (MODE == kModeSqrt && p.active && p.active[b] == 0) {
      if (threadIdx.x == 0) {
        p.info[b] = 0;
        if (p.iters) p.iters[b] = 0;
      }
      continue;
    }
    if (MODE == kModeExecute) run_execute(ops, p, b, n, off, M);
    if (MODE == kModePlan) run_plan(ops, p, b, n, off, M);
    if (MODE == kModeSqrt) run_sqrt(ops, p, b, n, off, M);
    if (MODE == kModeGraph) run_graph(ops, p, b, n, off, M);
    if (MODE == kModeBackward) run_backward(ops, p, b, n, off, W);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int small_kernel_slots(int count) {
  const int per_sm = LG_MINBLOCKS;  // blocks resident per SM (shared memory and registers)
  const int cap = lg::device_sm_count() * per_sm;
  return count < cap ? (count > 0 ? count : 1) : cap;
}

size_t small_order_bytes(int count) {
  const size_t raw = sizeof(int32_t) * ((size_t)count + 2 * kOrderBuckets + (size_t)count);
  return (raw + 255) / 256 * 256;
}

size_t small_bwd_workspace_bytes(int count, int n_max) {
  const size_t slots = (size_t)small_kernel_slots(count);
  return 256 + small_order_bytes(count) + slots * kBwdSlotMats * (size_t)n_max * n_max * sizeof(double) +
         slots * kBwdTapeCap * sizeof(double);
}

size_t small_workspace_bytes(int count, int n_max) {
  const size_t slots = (size_t)small_kernel_slots(count);
  return 256 + small_order_bytes(count) + slots * kSlotMats * (size_t)n_max * n_max * sizeof(double);
}

template <int MODE>
static cudaError_t launch_mode(const SmallParams& p, cudaStream_t st) {
  static lg::DeviceOnce attr;
  // shared memory: BlockSmem, plus the slot's kSlotMats matrices in the
  // shared-memory slot mode (the attribute allows the configuration's largest n)
  const size_t smem_cap = smem_slot<MODE>() ? kSmemSlotOffset + sizeof(double) * kSlotMats * kMaxN * kMaxN
                                            : sizeof(BlockSmem);
  const size_t smem = smem_slot<MODE>()
                          ? kSmemSlotOffset + sizeof(double) * kSlotMats * (size_t)p.n_max * p.n_max
                          : sizeof(BlockSmem);
  cudaError_t e = attr.run([&] {
    return cudaFuncSetAttribute(k_logm_small<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap);
  });
  if (e != cudaSuccess) return e;
  SmallParams q = p;
  if (smem_slot<MODE>()) {
    // as many persistent blocks as fit with this n_max's slot (no workspace slots)
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_logm_small<MODE>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const int cap = per_sm * lg::device_sm_count();
    q.n_slots = p.count < cap ? p.count : cap;
  }
  e = cudaMemsetAsync(p.queue, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  if (MODE == kModeExecute && p.order && p.order_aux && p.count > 1) {
    e = cudaMemsetAsync(p.order_aux, 0, sizeof(int32_t) * 2 * kOrderBuckets, st);
    if (e != cudaSuccess) return e;
    const int kb = p.count < 4 * lg::device_sm_count() ? p.count : 4 * lg::device_sm_count();
    k_order_keys<<<kb, kThreads, 0, st>>>(p);
    k_order_scan<<<1, 32, 0, st>>>(p);
    k_order_scatter<<<(p.count + kThreads - 1) / kThreads, kThreads, 0, st>>>(p);
  }
  if (!(MODE == kModeExecute && p.count > 1)) q.order = nullptr;
  k_logm_small<MODE><<<q.n_slots, kThreads, smem, st>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_small(Mode mode, const SmallParams& p, cudaStream_t st) {
  if (p.count <= 0) return cudaSuccess;
  switch (mode) {
    case kModeExecute: return launch_mode<kModeExecute>(p, st);
    case kModePlan: return launch_mode<kModePlan>(p, st);
    case kModeSqrt: return launch_mode<kModeSqrt>(p, st);
    case kModeGraph: return launch_mode<kModeGraph>(p, st);
    case kModeBackward: return launch_mode<kModeBackward>(p, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace LG_NS
