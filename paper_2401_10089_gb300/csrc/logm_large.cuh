// logm_large.cuh -- the whole-GPU kernel (n > kSmallMaxN) and its launcher
// template. Each (mode, update path) instantiation is compiled in its own
// translation unit (logm_large_*.cu) so that the build runs them in
// parallel; logm_large.cu holds the dispatcher.
//
// Algorithm 1 of arXiv 2401.10089 (Sec. 6) with the whole
// GPU on one matrix at a time, for n > kSmallMaxN (e.g. one 4096 x 4096
// matrix). A single cooperative launch (all blocks resident) walks the batch;
// the plan, the Denman-Beavers square roots (Gauss-Jordan inverses spread over
// all SMs) and the graph products all run inside it, separated by bounded
// grid barriers, with no host round trip.
#pragma once

#include <cuda.h>

#include <cmath>
#include <cstring>

#include "grid_ops.cuh"
#include "logm_algo.cuh"
#include "logm_internal.h"

namespace lg {

// SLICED: the Gauss-Jordan updates run on the tensor cores (tc_update.cuh);
// one block per SM then (its shared memory holds the digit tiles and it owns
// all 512 TMEM columns, allocated here for the whole launch).
template <int MODE, bool SLICED>
__global__ void __launch_bounds__(kThreads, SLICED ? 1 : 2)
    k_logm_large(SmallParams p, GridWs w, Slot M, const __grid_constant__ SliceMaps maps) {
  __shared__ GridSmem S;
  if (threadIdx.x == 0) {
    S.ep[0] = S.ep[1] = S.ep[2] = 0;
    if (SLICED) {
      for (int t = 0; t < kUpdStages; ++t) {
        tm_bar_init(su32(&S.slc.full[t]), 1);
        tm_bar_init(su32(&S.slc.empty[t]), 1);
      }
      tm_bar_init(su32(&S.slc.acc), 1);
      S.slc.stages = 0;
      S.slc.tiles = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (SLICED && threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.slc.tmem)),
                 "r"(kUpdTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  GridOps ops{w, S, 0, SLICED ? &maps : nullptr};
  for (int b = 0; b < p.count; ++b) {
    int n;
    int64_t off;
    matrix_geometry(p, b, &n, &off);
    if (n <= kSmallMaxN && p.large_pass) continue;  // handled by the one-block-per-matrix kernel
    if (n < 1 || n > p.n_max) {
      if (ops.leader()) {
        if (p.info) p.info[b] = -1;
        if (p.s_out) p.s_out[b] = 0;
        if (p.k_out) p.k_out[b] = p.k_max;
      }
      continue;
    }
    if (MODE == kModeSqrt && p.active && p.active[b] == 0) {
      if (ops.leader()) {
        p.info[b] = 0;
        if (p.iters) p.iters[b] = 0;
      }
      continue;
    }
    if (MODE == kModeExecute) run_execute(ops, p, b, n, off, M);
    if (MODE == kModePlan) run_plan(ops, p, b, n, off, M);
    if (MODE == kModeSqrt) run_sqrt(ops, p, b, n, off, M);
    if (MODE == kModeGraph) run_graph(ops, p, b, n, off, M);
    ops.sync();
    if (ops.leader() && *(volatile int*)w.err && p.info) p.info[b] = 5;  // barrier timed out
  }
  if (SLICED) {
    tm_fence_before();
    __syncthreads();
    if (threadIdx.x < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.slc.tmem), "r"(kUpdTmemCols));
  }
}

namespace large_detail {

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct GroupLayout {
  size_t cand_v, cand_i, cand_row, row_k, pivval, ldpart, panel, R, piv, perm, work, adig, bdig, aexp, bexp, ucat,
      vcat;
};

struct LargeLayout {
  size_t bar, partial, ipartial, vec, colpart, misc, slot, total;
  GroupLayout g[2];
};

inline LargeLayout large_layout(int n_max) {
  LargeLayout L{};
  size_t o = 0;
  const size_t nm = (size_t)n_max;
  L.bar = o;      o = align256(o + 64);  // main barrier counter, error word, two group barrier counters
  L.partial = o;  o = align256(o + sizeof(double) * 2 * kMaxGrid);
  L.ipartial = o; o = align256(o + sizeof(int) * 2 * kMaxGrid);
  L.vec = o;      o = align256(o + sizeof(double) * 4 * nm);
  L.colpart = o;  o = align256(o + sizeof(double) * 2 * kColGroups * nm);
  L.misc = o;     o = align256(o + sizeof(double) * 16);
  for (int t = 0; t < 2; ++t) {
    GroupLayout& g = L.g[t];
    g.cand_v = o; o = align256(o + sizeof(unsigned long long) * 2 * kMaxGrid);
    g.cand_i = o; o = align256(o + sizeof(int) * 2 * kMaxGrid);
    g.cand_row = o; o = align256(o + sizeof(double) * 2 * kMaxGrid * kGridPanel);
    g.row_k = o;  o = align256(o + sizeof(double) * 2 * kGridPanel);
    g.pivval = o; o = align256(o + sizeof(double) * nm);
    g.ldpart = o; o = align256(o + sizeof(double) * kMaxGrid);
    g.panel = o;  o = align256(o + sizeof(double) * kGridPanel * nm);
    g.R = o;      o = align256(o + sizeof(double) * kGridPanel * nm);
    g.piv = o;    o = align256(o + sizeof(int) * nm);
    g.perm = o;   o = align256(o + sizeof(int) * nm);
    g.work = o;   o = align256(o + sizeof(double) * nm * nm);
    g.adig = o;   o = align256(o + 2 * (size_t)kDigRow * nm);  // BF16 digits of the tensor-core updates
    g.bdig = o;   o = align256(o + 2 * (size_t)kDigRow * nm);
    g.aexp = o;   o = align256(o + sizeof(int32_t) * nm);
    g.bexp = o;   o = align256(o + sizeof(int32_t) * nm);
    g.ucat = o;   o = align256(o + sizeof(double) * kSuperCols * nm);  // deferred factors of a super-panel
    g.vcat = o;   o = align256(o + sizeof(double) * kSuperCols * nm);
  }
  L.slot = o;     o = align256(o + sizeof(double) * kSlotMats * nm * nm);
  L.total = o;
  return L;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn tensor_map_encoder() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(f);
    return static_cast<EncodeTiledFn>(nullptr);
  }();
  return fn;
}

// 3-D map over a digit buffer of n_max rows of kDigRow BF16, read as
// (term within a group of gx, row, group): box gx x box_rows x box_groups,
// 128-byte (gx = 64) or 32-byte (gx = 16) swizzle, zero fill outside. The
// copy lands in shared memory group-major: [group][row][gx terms].
inline bool digit_map(CUtensorMap* m, void* base, int n_max, int gx, int box_rows, int box_groups) {
  EncodeTiledFn f = tensor_map_encoder();
  if (!f) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)gx, (cuuint64_t)n_max, (cuuint64_t)(kDigRow / gx)};
  const cuuint64_t strides[2] = {(cuuint64_t)kDigRow * 2, (cuuint64_t)gx * 2};
  const cuuint32_t box[3] = {(cuuint32_t)gx, (cuuint32_t)box_rows, (cuuint32_t)box_groups};
  const cuuint32_t estr[3] = {1, 1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           gx == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, bool SLICED>
cudaError_t launch_large_mode(const SmallParams& p, char* ws, cudaStream_t st) {
  const LargeLayout L = large_layout(p.n_max);
  GridWs w{};
  w.bar = reinterpret_cast<unsigned long long*>(ws + L.bar);
  w.err = reinterpret_cast<int*>(ws + L.bar + 8);
  w.partial = reinterpret_cast<double*>(ws + L.partial);
  w.ipartial = reinterpret_cast<int*>(ws + L.ipartial);
  w.vec = reinterpret_cast<double*>(ws + L.vec);
  w.colpart = reinterpret_cast<double*>(ws + L.colpart);
  w.misc = reinterpret_cast<double*>(ws + L.misc);
  for (int t = 0; t < 2; ++t) {
    GjGroup& g = w.gj[t];
    const GroupLayout& gl = L.g[t];
    g.bar = reinterpret_cast<unsigned long long*>(ws + L.bar + 16 + 8 * t);
    g.cand_v = reinterpret_cast<unsigned long long*>(ws + gl.cand_v);
    g.pivval = reinterpret_cast<double*>(ws + gl.pivval);
    g.ldpart = reinterpret_cast<double*>(ws + gl.ldpart);
    g.cand_i = reinterpret_cast<int*>(ws + gl.cand_i);
    g.cand_row = reinterpret_cast<double*>(ws + gl.cand_row);
    g.row_k = reinterpret_cast<double*>(ws + gl.row_k);
    g.panel = reinterpret_cast<double*>(ws + gl.panel);
    g.R = reinterpret_cast<double*>(ws + gl.R);
    g.piv = reinterpret_cast<int*>(ws + gl.piv);
    g.perm = reinterpret_cast<int*>(ws + gl.perm);
    g.work = reinterpret_cast<double*>(ws + gl.work);
    g.result = w.misc + 8 + 2 * t;
    g.sl.adig = reinterpret_cast<__nv_bfloat16*>(ws + gl.adig);
    g.sl.bdig = reinterpret_cast<__nv_bfloat16*>(ws + gl.bdig);
    g.sl.aexp = reinterpret_cast<int32_t*>(ws + gl.aexp);
    g.sl.bexp = reinterpret_cast<int32_t*>(ws + gl.bexp);
    g.ucat = reinterpret_cast<double*>(ws + gl.ucat);
    g.vcat = reinterpret_cast<double*>(ws + gl.vcat);
    g.gi = t;
  }
  SliceMaps maps;
  memset(&maps, 0, sizeof(maps));
  if (SLICED)
    for (int t = 0; t < 2; ++t)
      if (!digit_map(&maps.a[t], ws + L.g[t].adig, p.n_max, 64, kUpdM, 2) ||
          !digit_map(&maps.b[t], ws + L.g[t].bdig, p.n_max, 16, kUpdN, kSlices))
        return cudaErrorNotSupported;
  w.n_max = p.n_max;
  const int64_t nn = (int64_t)p.n_max * p.n_max;
  double* base = reinterpret_cast<double*>(ws + L.slot);
  Slot M{base, base + nn, base + 2 * nn, base + 3 * nn, base + 4 * nn, base + 5 * nn, base + 6 * nn};

  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // Dynamic shared memory: two buffers of a block's panel rows, sized for the
  // smallest group (half the grid), and at least the DMMA tiles of the FP64
  // products; with SLICED also the transposed factor rows of a super-panel,
  // and at least the stage ring and staged tile of the tensor-core updates
  // (which also keeps one block per SM, the owner of its SM's TMEM). Two
  // blocks per SM if they fit, else one.
  int grid = 0;
  size_t dyn = 0;
  for (int want = SLICED ? 1 : 2; want >= 1 && grid == 0; --want) {
    int gsz = sms * want;
    if (gsz > kMaxGrid) gsz = kMaxGrid;
    const int min_group = gsz / 2 >= 8 ? gsz / 2 : gsz;
    size_t d = 2 * (size_t)((p.n_max + min_group - 1) / min_group) * kSpStride * sizeof(double);
    if (SLICED) d += sizeof(double) * (kSuperCols - kGridPanel) * kGridPanel;
    if (d < sizeof(GemmSmem)) d = sizeof(GemmSmem);
    if (SLICED && d < kUpdSmemBytes) d = kUpdSmemBytes;
    e = cudaFuncSetAttribute(k_logm_large<MODE, SLICED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d);
    if (e != cudaSuccess) continue;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_logm_large<MODE, SLICED>, kThreads, d);
    if (e != cudaSuccess) return e;
    if (per_sm >= want && (!SLICED || per_sm == 1)) {
      grid = gsz;
      dyn = d;
    }
  }
  if (grid < 1) return cudaErrorLaunchOutOfResources;

  e = cudaMemsetAsync(ws + L.bar, 0, 64, st);
  if (e != cudaSuccess) return e;
  if (SLICED)  // digit rows past a matrix's n are never written: they stay zero
    for (int t = 0; t < 2; ++t) {
      e = cudaMemsetAsync(ws + L.g[t].adig, 0, L.g[t].ucat - L.g[t].adig, st);
      if (e != cudaSuccess) return e;
    }
  SmallParams pp = p;
  void* args[] = {&pp, &w, &M, &maps};
  return cudaLaunchCooperativeKernel((const void*)k_logm_large<MODE, SLICED>, dim3(grid), dim3(kThreads), args, dyn,
                                     st);
}

}  // namespace large_detail

}  // namespace lg
