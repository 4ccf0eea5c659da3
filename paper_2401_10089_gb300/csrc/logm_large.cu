// logm_large.cu -- Algorithm 1 of arXiv 2401.10089 (Sec. 6) with the whole
// GPU on one matrix at a time, for n > kSmallMaxN (e.g. one 4096 x 4096
// matrix). A single cooperative launch (all blocks resident) walks the batch;
// the plan, the Denman-Beavers square roots (Gauss-Jordan inverses spread over
// all SMs) and the graph products all run inside it, separated by bounded
// grid barriers, with no host round trip.
#include <cmath>

#include "grid_ops.cuh"
#include "logm_algo.cuh"
#include "logm_internal.h"

namespace lg {

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_logm_large(SmallParams p, GridWs w, Slot M) {
  __shared__ GridSmem S;
  if (threadIdx.x == 0) S.ep[0] = S.ep[1] = S.ep[2] = 0;
  __syncthreads();
  GridOps ops{w, S, 0};
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
}

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct GroupLayout {
  size_t cand_v, cand_i, cand_row, row_k, pivval, ldpart, panel, R, piv, perm, work;
};

struct LargeLayout {
  size_t bar, partial, ipartial, vec, colpart, misc, slot, total;
  GroupLayout g[2];
};

LargeLayout large_layout(int n_max) {
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
  }
  L.slot = o;     o = align256(o + sizeof(double) * kSlotMats * nm * nm);
  L.total = o;
  return L;
}

template <int MODE>
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
  }
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
  // smallest group (half the grid). Two blocks per SM if they fit, else one.
  int grid = 0;
  size_t dyn = 0;
  for (int want = 2; want >= 1 && grid == 0; --want) {
    int gsz = sms * want;
    if (gsz > kMaxGrid) gsz = kMaxGrid;
    const int min_group = gsz / 2 >= 8 ? gsz / 2 : gsz;
    const size_t d = 2 * (size_t)((p.n_max + min_group - 1) / min_group) * kGridPanel * sizeof(double);
    e = cudaFuncSetAttribute(k_logm_large<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d);
    if (e != cudaSuccess) continue;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_logm_large<MODE>, kThreads, d);
    if (e != cudaSuccess) return e;
    if (per_sm >= want) {
      grid = gsz;
      dyn = d;
    }
  }
  if (grid < 1) return cudaErrorLaunchOutOfResources;

  e = cudaMemsetAsync(ws + L.bar, 0, 64, st);
  if (e != cudaSuccess) return e;
  SmallParams pp = p;
  void* args[] = {&pp, &w, &M};
  return cudaLaunchCooperativeKernel((const void*)k_logm_large<MODE>, dim3(grid), dim3(kThreads), args, dyn, st);
}

}  // namespace

size_t large_workspace_bytes(int n_max) { return large_layout(n_max).total; }

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
  switch (mode) {
    case kModeExecute: return launch_large_mode<kModeExecute>(p, w, st);
    case kModePlan: return launch_large_mode<kModePlan>(p, w, st);
    case kModeSqrt: return launch_large_mode<kModeSqrt>(p, w, st);
    case kModeGraph: return launch_large_mode<kModeGraph>(p, w, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lg
