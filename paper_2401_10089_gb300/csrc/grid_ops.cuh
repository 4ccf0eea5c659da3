// grid_ops.cuh -- the whole-GPU ops layer for one large matrix at a time.
//
// One cooperative launch (every block resident) runs Algorithm 1 with all
// blocks working on the same matrix; phases are separated by a grid barrier.
// The barrier is a monotonic 64-bit arrival counter (no reset: episode e of a
// barrier completes when its counter reaches (e + 1) * nblocks; each block
// counts its episodes in shared memory), one release add and acquire polls.
// It is bounded: a block that waits longer than kBarrierTimeoutNs sets an
// error flag, and from then on every barrier returns at once, so the kernel
// always finishes (with LOGM_INFO error status) instead of hanging.
//
// Reductions are deterministic and identical in every block: each block
// writes its partial result, and after the barrier every block reduces the
// same array in the same order. That keeps every branch of Algorithm 1
// uniform across the grid.
#pragma once

#include <cstdint>

#include "cta_linalg.cuh"
#include "tc_update.cuh"

namespace lg {

constexpr int kGridPanel = 32;          // Gauss-Jordan panel width for large n
constexpr int kSpStride = kGridPanel + 1;  // doubles per row of a panel in shared memory (column walks conflict-free)
constexpr int kSuperCols = kMaxChunks * kGridPanel;  // tensor-core form: columns of a super-panel
static_assert(kGridPanel == kSliceK, "a panel is one chunk of the tensor-core updates");
constexpr int kColGroups = 16;          // row groups of the column passes (norms, transposed mat-vecs, updates)
constexpr int kMaxGrid = 1024;          // upper bound on co-resident blocks
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;  // 20 s
constexpr unsigned long long kBarrierMaxPolls = 1ull << 26;  // backstop should the clock not advance

// Buffers of one Gauss-Jordan inversion running on a group of blocks.
struct GjGroup {
  unsigned long long* bar;  // arrival counter of the group's own barrier
  unsigned long long* cand_v;  // [2][kMaxGrid] pivot candidates: |value| as an ordered integer key
  int* cand_i;       // [2][kMaxGrid] pivot candidates (row)
  double* pivval;    // [n_max] pivot of every Gauss-Jordan step (log|det| is summed after the loop)
  double* ldpart;    // [kMaxGrid] per-block partial sums of log|pivot|
  double* cand_row;  // [2][kMaxGrid][kGridPanel] each block's candidate row of the panel
  double* row_k;     // [2][kGridPanel] the panel row of the next pivot position
  double* panel;     // [kGridPanel][n_max] the finished panel, column-major
  double* R;         // [kGridPanel][n_max] pivot rows of the panel
  int* piv;          // [n_max] pivot rows of the Gauss-Jordan steps
  int* perm;         // [n_max] composite column permutation
  double* work;      // [n_max^2] working matrix
  double* result;    // [2] log|det|, status
  SliceBufs sl;      // tensor-core updates: digits of the factors
  double* ucat;      // [n_max][kSuperCols] tensor-core form: the factors U_q of a super-panel's sub-panels
  double* vcat;      // [n_max][kSuperCols] tensor-core form: their pivot rows v_q, by column
  int gi;            // index of this group (its tensor maps)
};

struct GridWs {
  unsigned long long* bar;  // arrival counter of the whole-grid barrier (zeroed before the launch)
  int* err;          // set when a barrier wait timed out (zeroed before the launch)
  double* partial;   // [2][kMaxGrid] partial results of sum / max
  int* ipartial;     // [2][kMaxGrid] partial results of all / argmax indices
  double* vec;       // [4][n_max] estimator vectors
  double* colpart;   // [2][kColGroups][n_max] partial column sums of the column passes
  double* misc;      // [8] broadcast slots
  GjGroup gj[2];     // the two inversion groups (gj[0] alone when one inversion uses the whole grid)
  int n_max;
};

struct GridSmem {
  Reduce red;
  double rowk[kGridPanel];
  double rowp[kGridPanel];
  double prow[kGridPanel];
  double bc[4];
  int work[4];
  unsigned long long ep[3];  // barrier episodes seen: whole grid, group 0, group 1
  int pivot_row;             // pivot row of the current Gauss-Jordan column (-1: no valid pivot)
  SliceSmem slc;             // tensor-core updates: barriers, phases, TMEM base
  int skip_upd;              // the grid's error word was set: no more tensor-core work
  int psrc[2 * kGridPanel];  // rows traced back through a panel's swaps
  int ppos[2 * kGridPanel];  // the positions they move to
};

// Geometry of one Gauss-Jordan inversion on a group of G blocks: this block's
// index in the group (lb), its thread index in the group (gt of gnt), its rows
// [r_lo, r_hi) of rows_per, its two panel buffers in shared memory, and the
// group's barrier counter and this block's episode count of it.
struct GjCtx {
  int lb, gt, gnt, G, rows_per, r_lo, r_hi, my_rows;
  double* Sp0;
  double* Sp1;
  unsigned long long* bar;
  unsigned long long* ep;
};

// Dynamic shared memory of the whole-GPU kernel, used by one phase at a time:
// this block's rows of the current Gauss-Jordan panel (row-major, two buffers
// of rows_per x kSpStride) and, in the tensor-core form, the transposed rows
// of the earlier sub-panels' factors after them; the stage ring and staged
// tile of the tensor-core updates; the DMMA tiles of the FP64-pipe products.
extern __shared__ double grid_panel_smem[];

static __device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

static __device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

static __device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Barrier over `nblocks` blocks sharing the arrival counter *bar; *ep is this
// block's episode count for that counter (shared memory, thread 0 only).
// Gives up after timeout_ns (or kBarrierMaxPolls polls), setting *err = 1.
static __device__ void bounded_barrier(unsigned long long* bar, unsigned nblocks, int* err,
                                       unsigned long long* ep,
                                       unsigned long long timeout_ns = kBarrierTimeoutNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* verr = err;
    const unsigned long long target = (*ep + 1) * nblocks;
    *ep += 1;
    if (*verr == 0) {
      red_release_add(bar, 1ull);  // publishes this block's writes (release, gpu scope)
      const unsigned long long t0 = global_ns();
      unsigned long long polls = 0;
      while (ld_acquire(bar) < target) {
        if (*verr) break;
        ++polls;
        if (((polls & 63) == 0 && global_ns() - t0 > timeout_ns) || polls > kBarrierMaxPolls) {
          atomicExch(err, 1);
          break;
        }
      }
    }
  }
  // the acquire load that saw every arrival orders thread 0 after the other
  // blocks' releases; the block barrier orders the other threads after it
  __syncthreads();
}

// bounded_barrier in two halves, so that a block can work between its
// arrival and the wait: barrier_arrive publishes the block's writes (block
// barrier, then thread 0's release add), barrier_wait polls for the others
// (the same bound) and ends with a block barrier.
static __device__ void barrier_arrive(unsigned long long* bar, unsigned nblocks, int* err, unsigned long long* ep) {
  __syncthreads();
  if (threadIdx.x == 0) {
    *ep += 1;
    if (*(volatile int*)err == 0) red_release_add(bar, 1ull);
  }
}
static __device__ void barrier_wait(unsigned long long* bar, unsigned nblocks, int* err, unsigned long long* ep,
                                    unsigned long long timeout_ns = kBarrierTimeoutNs) {
  if (threadIdx.x == 0) {
    volatile int* verr = err;
    const unsigned long long target = *ep * nblocks;
    if (*verr == 0) {
      const unsigned long long t0 = global_ns();
      unsigned long long polls = 0;
      while (ld_acquire(bar) < target) {
        if (*verr) break;
        ++polls;
        if (((polls & 63) == 0 && global_ns() - t0 > timeout_ns) || polls > kBarrierMaxPolls) {
          atomicExch(err, 1);
          break;
        }
      }
    }
  }
  __syncthreads();
}

struct GridOps {
  GridWs& w;
  GridSmem& S;
  int rbuf;  // alternating partial buffer of the generic reductions
  const SliceMaps* maps;  // non-null: the Gauss-Jordan updates run on the tensor cores (tc_update.cuh)

  __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ int nthreads() const { return gridDim.x * blockDim.x; }
  __device__ void sync() { bounded_barrier(w.bar, gridDim.x, w.err, &S.ep[0]); }
  __device__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
  __device__ GemmSmem& gsm() const { return *reinterpret_cast<GemmSmem*>(grid_panel_smem); }

  __device__ double sum(double v) {
    const double bs = block_sum(v, S.red);
    double* part = w.partial + rbuf * kMaxGrid;
    rbuf ^= 1;
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    sync();
    double t = 0.0;
    for (int g = threadIdx.x; g < (int)gridDim.x; g += kThreads) t += part[g];
    return block_sum(t, S.red);
  }

  __device__ double max(double v) {
    const double bm = block_max(v, S.red);
    double* part = w.partial + rbuf * kMaxGrid;
    rbuf ^= 1;
    if (threadIdx.x == 0) part[blockIdx.x] = bm;
    sync();
    double t = 0.0;
    for (int g = threadIdx.x; g < (int)gridDim.x; g += kThreads) t = nanmax(t, part[g]);
    return block_max(t, S.red);
  }

  __device__ int all(int v) {
    const int ba = block_and(v, S.red);
    int* part = w.ipartial + rbuf * kMaxGrid;
    rbuf ^= 1;
    if (threadIdx.x == 0) part[blockIdx.x] = ba;
    sync();
    int t = 1;
    for (int g = threadIdx.x; g < (int)gridDim.x; g += kThreads) t &= part[g];
    return block_and(t, S.red);
  }

  __device__ void argmax(double v, int i, double* ov, int* oi) {
    double bv;
    int bi;
    block_argmax(v, i, S.red, &bv, &bi);
    double* pv = w.partial + rbuf * kMaxGrid;
    int* pi = w.ipartial + rbuf * kMaxGrid;
    rbuf ^= 1;
    if (threadIdx.x == 0) {
      pv[blockIdx.x] = bv;
      pi[blockIdx.x] = bi;
    }
    sync();
    double cv = -1.0;
    int ci = 0x7fffffff;
    for (int g = threadIdx.x; g < (int)gridDim.x; g += kThreads)
      if (pv[g] > cv || (pv[g] == cv && pi[g] < ci)) {
        cv = pv[g];
        ci = pi[g];
      }
    block_argmax(cv, ci, S.red, ov, oi);
  }

  __device__ double bcast0(double v) {
    if (threadIdx.x == 0) S.bc[0] = v;
    __syncthreads();
    const double r = S.bc[0];
    __syncthreads();
    return r;
  }

  __device__ double* vec(int i) { return w.vec + (int64_t)i * w.n_max; }

  // Column passes: with n columns and T threads, thread t takes column t % n
  // and every R-th row from t / n (R = min(kColGroups, T / n) row groups), so
  // that all threads work (one thread per column would leave most of a grid
  // idle for n of a few thousand); the R partial sums per column meet in
  // w.colpart after one barrier.
  __device__ int col_groups(int n) const {
    const int r = nthreads() / n;
    return r < 1 ? 1 : (r > kColGroups ? kColGroups : r);
  }

  __device__ double norm1(const double* M, int n, double shift) {
    const int R = col_groups(n), t = tid();
    if (t < n * R) {
      const int j = t % n, r = t / n;
      double s = 0.0;
      for (int i = r; i < n; i += R) {
        double v = M[(int64_t)i * n + j];
        if (i == j) v -= shift;
        s += fabs(v);
      }
      w.colpart[(int64_t)r * n + j] = s;
    }
    sync();
    double best = 0.0;
    for (int j = t; j < n; j += nthreads()) {
      double s = 0.0;
      for (int r = 0; r < R; ++r) s += w.colpart[(int64_t)r * n + j];
      best = nanmax(best, s);
    }
    return max(best);
  }

  // Denman-Beavers update, eq. (ScalDB): X <- (mu X + Yi / mu) / 2, Y <- (mu Y +
  // Xi / mu) / 2; returns ||X_new - X_old||_1 and ||X_new||_1.
  __device__ void db_update(double* X, double* Y, const double* Xi, const double* Yi, double mu, double imu, int n,
                            double* nd, double* nx) {
    const int R = col_groups(n), t = tid();
    double* cd_part = w.colpart;
    double* cx_part = w.colpart + (int64_t)kColGroups * w.n_max;
    if (t < n * R) {
      const int j = t % n, r = t / n;
      double cd = 0.0, cx = 0.0;
      for (int i = r; i < n; i += R) {
        const int64_t q = (int64_t)i * n + j;
        const double xo = X[q];
        const double xn = 0.5 * fma(mu, xo, Yi[q] * imu);
        Y[q] = 0.5 * fma(mu, Y[q], Xi[q] * imu);
        X[q] = xn;
        cd += fabs(xn - xo);
        cx += fabs(xn);
      }
      cd_part[(int64_t)r * n + j] = cd;
      cx_part[(int64_t)r * n + j] = cx;
    }
    sync();
    double sd = 0.0, sx = 0.0;
    for (int j = t; j < n; j += nthreads()) {
      double cd = 0.0, cx = 0.0;
      for (int r = 0; r < R; ++r) {
        cd += cd_part[(int64_t)r * n + j];
        cx += cx_part[(int64_t)r * n + j];
      }
      sd = nanmax(sd, cd);
      sx = nanmax(sx, cx);
    }
    *nd = max(sd);
    *nx = max(sx);
  }

  // Product-form update: X <- (mu X + XMi / mu) / 2 (XMi = I in the first step),
  // M <- M^{-1}/(4 mu^2) + mu^2 M / 4 + I/2; returns ||X_new - X_old||_1, ||X_new||_1.
  __device__ void db_update_product(double* X, double* Mk, const double* Mi, const double* XMi, bool first,
                                    double mu, double imu, double mu2, double imu2, int n, double* nd, double* nx) {
    const int R = col_groups(n), t = tid();
    double* cd_part = w.colpart;
    double* cx_part = w.colpart + (int64_t)kColGroups * w.n_max;
    if (t < n * R) {
      const int j = t % n, r = t / n;
      double cd = 0.0, cx = 0.0;
      for (int i = r; i < n; i += R) {
        const int64_t q = (int64_t)i * n + j;
        const double xo = X[q];
        const double xmi = first ? (i == j ? 1.0 : 0.0) : XMi[q];
        const double xn = 0.5 * fma(mu, xo, xmi * imu);
        Mk[q] = fma(0.25, fma(mu2, Mk[q], Mi[q] * imu2), i == j ? 0.5 : 0.0);
        X[q] = xn;
        cd += fabs(xn - xo);
        cx += fabs(xn);
      }
      cd_part[(int64_t)r * n + j] = cd;
      cx_part[(int64_t)r * n + j] = cx;
    }
    sync();
    double sd = 0.0, sx = 0.0;
    for (int j = t; j < n; j += nthreads()) {
      double cd = 0.0, cx = 0.0;
      for (int r = 0; r < R; ++r) {
        cd += cd_part[(int64_t)r * n + j];
        cx += cx_part[(int64_t)r * n + j];
      }
      sd = nanmax(sd, cd);
      sx = nanmax(sx, cx);
    }
    *nd = max(sd);
    *nx = max(sx);
  }

  __device__ void matvec(const double* M, int n, double shift, const double* x, double* y, int trans) {
    if (!trans) {
      const int lane = threadIdx.x & 31;
      const int gw = tid() >> 5, nw = nthreads() >> 5;
      for (int i = gw; i < n; i += nw) {
        double s = 0.0;
        const double* row = M + (int64_t)i * n;
        for (int c = lane; c < n; c += 32) s = fma(row[c], x[c], s);
        s = warp_sum(s);
        if (lane == 0) y[i] = s - shift * x[i];
      }
    } else {
      // y = M^T x - shift x as a column pass: partial sums over row groups
      const int R = col_groups(n), t = tid();
      if (t < n * R) {
        const int j = t % n, r = t / n;
        double s0 = 0.0;
        for (int i = r; i < n; i += R) s0 = fma(M[(int64_t)i * n + j], x[i], s0);
        w.colpart[(int64_t)r * n + j] = s0;
      }
      sync();
      for (int j = t; j < n; j += nthreads()) {
        double s0 = 0.0;
        for (int r = 0; r < R; ++r) s0 += w.colpart[(int64_t)r * n + j];
        y[j] = s0 - shift * x[j];
      }
    }
    sync();
  }

  __device__ void gemm(int n, const double* A, double as, const double* B, double bs, double alpha,
                       const EpiTerms& e, OutView out, bool ta = false, bool tb = false) {
    if (maps && !ta && !tb) {
      gemm_sliced(n, A, as, B, bs, alpha, e, out);
      return;
    }
    const int tiles = (n + kTileM - 1) / kTileM;
    for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x)
      gemm_tile(n, (t / tiles) * kTileM, (t % tiles) * kTileN, A, as, B, bs, alpha, e, out, gsm(), ta, tb);
    sync();
  }

  // out = alpha (A - as I)(B - bs I) + sum_t e.c[t] e.M[t] on the tensor cores:
  // K in chunks of kSuperCols, each chunk's product formed exactly from BF16
  // digits (tc_update.cuh, per-row scales of the chunk of A, per-column scales
  // of the chunk of B) and added to an FP64 accumulator, then the epilogue
  // terms. Uses group 0's digit buffers and working matrix (free outside the
  // inversions) with every block of the grid.
  __device__ __noinline__ void gemm_sliced(int n, const double* A, double as, const double* B, double bs, double alpha,
                              const EpiTerms& e, OutView out) {
    GjGroup& g = w.gj[0];
    double* C = g.work;
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = tid(); t < nn; t += nthreads()) C[t] = 0.0;
    const int ncb = (n + kUpdN - 1) / kUpdN;
    const int T = ((n + kUpdM - 1) / kUpdM) * ncb;
    const int G = gridDim.x, lb = blockIdx.x;
    const int t_lo = (int)((int64_t)lb * T / G), t_hi = (int)((int64_t)(lb + 1) * T / G);
    for (int kb = 0; kb < n; kb += kSuperCols) {
      const int jb = min(kSuperCols, n - kb), nc = (jb + kSliceK - 1) / kSliceK;
      // digits of A[:, kb..kb+jb) by rows (rc < n) and of B[kb..kb+jb, :] by
      // columns (rc - n), eight lanes per row or column, four per warp at a time
      {
        const int lane = threadIdx.x & 31, i = lane & 7;
        const int gw = tid() >> 5, nw = nthreads() >> 5;
        for (int q4 = gw * 4; q4 < 2 * n; q4 += nw * 4) {
          const int rc = q4 + (lane >> 3);
          const bool valid = rc < 2 * n, isa = rc < n;
          double u[4 * kMaxChunks];
#pragma unroll
          for (int c = 0; c < kMaxChunks; ++c)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int kk = kSliceK * c + 4 * i + t;
              double x = 0.0;
              if (valid && kk < jb) {
                if (isa)
                  x = A[(int64_t)rc * n + kb + kk] - (rc == kb + kk ? as : 0.0);
                else
                  x = B[(int64_t)(kb + kk) * n + (rc - n)] - (kb + kk == rc - n ? bs : 0.0);
              }
              u[4 * c + t] = x;
            }
          const int64_t row = !valid ? 0 : isa ? rc : rc - n;
          slice_row8<kMaxChunks>(u, i, valid, nc, (isa ? g.sl.adig : g.sl.bdig) + row * kDigRow,
                                 (isa ? g.sl.aexp : g.sl.bexp) + row);
        }
      }
      fence_proxy_async_global();
      sync();
      if (threadIdx.x == 0) S.skip_upd = *(volatile int*)w.err;
      __syncthreads();
      if (!S.skip_upd) {
        const UpdTiles ut{nc, 0, ncb, 1 << 30, 0, 0, 0};
        sliced_update(S.slc, reinterpret_cast<unsigned char*>(grid_panel_smem), &maps->a[0], &maps->b[0], g.sl, C, n,
                      ut, t_lo, t_hi, w.err);
      }
      sync();
    }
    for (int64_t t = tid(); t < nn; t += nthreads()) {
      double v = alpha * C[t];
      for (int s = 0; s < e.count; ++s) v = fma(e.c[s], e.M[s][t], v);
      store_out(out, (size_t)t, v);
    }
    sync();
  }

  __device__ void lincomb(int n, const EpiTerms& e, double* out) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = tid(); t < nn; t += nthreads()) {
      double v = 0.0;
      for (int s = 0; s < e.count; ++s) v = fma(e.c[s], e.M[s][t], v);
      out[t] = v;
    }
    sync();
  }

  // W[r0.., c0..] (64 x 64 tile) += (Pf - I_J)[r0.., 0..jb) R[0..jb), c0..], columns of J skipped.
  __device__ void rank_update_tile(double* W, int n, int kb, int jb, const double* Pf, const double* R, int r0,
                                   int c0) {
    GemmSmem& sm = gsm();
    const int tid_ = threadIdx.x, lane = tid_ & 31, warp = tid_ >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, q = lane & 3;
    double acc[2][4][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
    for (int k0 = 0; k0 < jb; k0 += kTileK) {
      for (int e = tid_; e < kTileM * kTileK; e += kThreads) {
        const int kk = e / kTileM, rr = e % kTileM;
        const int gr = r0 + rr, gk = k0 + kk;
        sm.As[rr * kAsStride + kk] = (gr < n && gk < jb) ? Pf[(int64_t)gk * n + gr] : 0.0;
      }
      for (int e = tid_; e < kTileK * kTileN; e += kThreads) {
        const int kk = e / kTileN, cc = e % kTileN;
        const int gk = k0 + kk, gc = c0 + cc;
        sm.Bs[kk * kBsStride + cc] = (gk < jb && gc < n) ? R[(int64_t)gk * n + gc] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < kTileK; ks += 4) {
        double af[2], bf[4];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) af[mb] = sm.As[(wm * 16 + mb * 8 + g) * kAsStride + ks + q];
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) bf[nb] = sm.Bs[(ks + q) * kBsStride + wn * 32 + nb * 8 + g];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
          for (int nb = 0; nb < 4; ++nb) dmma_8x8x4(acc[mb][nb][0], acc[mb][nb][1], af[mb], bf[nb]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
      for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int gr = r0 + wm * 16 + mb * 8 + g;
          const int gc = c0 + wn * 32 + nb * 8 + 2 * q + h;
          if (gr < n && gc < n && (gc < kb || gc >= kb + jb)) {
            double v = acc[mb][nb][h];
            if (gr >= kb && gr < kb + jb) v -= R[(int64_t)(gr - kb) * n + gc];  // the -I_J part
            W[(int64_t)gr * n + gc] += v;
          }
        }
  }

  // dst <- src^{-1} by Gauss-Jordan with partial pivoting (same steps as
  // gj_inverse_block), panels of kGridPanel columns, on the gn blocks
  // starting at g0 with the group's buffers, barrier counter `bar` and
  // episode count `ep`. The panel is spread over the group's blocks by rows
  // and each block keeps its rows in shared memory (grid_panel_smem, at most
  // rows_cap rows). Each column step is one group barrier: every block then
  // reads all blocks' pivot candidates and the row of the pivot position (one
  // round of loads), picks the pivot, reads the winning block's candidate row
  // (one more), applies the step to its own rows and publishes its candidate
  // for the next column together with that candidate's panel row. Writes
  // log|det| and the status (0, or 1 for a zero / non-finite pivot) to
  // g.result.
  // One Gauss-Jordan panel (columns [kb, kb + jb)) on the group: the block's
  // rows of W[:, J] into shared memory, then jb column steps (pivot search
  // over the group's candidates, scaled pivot row, elimination of the panel's
  // rows, the next column's candidates), one group barrier each. The finished
  // panel (this block's rows) is left in x.Sp1 if jb is odd, else x.Sp0; the
  // pivots in g.piv and g.pivval. Returns 1 for a zero or non-finite pivot.
  __device__ __noinline__ int panel_steps(GjGroup& g, const GjCtx& x, double* W, int n, int kb, int jb) {
    const int lb = x.lb, G = x.G, gn = x.G, rows_per = x.rows_per, r_lo = x.r_lo, r_hi = x.r_hi;
    const int my_rows = x.my_rows;
    double* Sp0 = x.Sp0;
    double* Sp1 = x.Sp1;
    unsigned long long* bar = x.bar;
    unsigned long long* ep = x.ep;
    const bool glead = lb == 0 && threadIdx.x == 0;
    // own rows of W[:, J] -> shared memory; candidates of column kb; the
    // candidate's row and the row of pivot position kb are published
    {
      unsigned long long cv = 0;
      int ci = 0x7fffffff;
      for (int e = threadIdx.x; e < my_rows * jb; e += kThreads) {
        const int rr = e / jb, c = e % jb;
        const int r = r_lo + rr;
        const double v = W[(int64_t)r * n + kb + c];
        Sp0[rr * kSpStride + c] = v;
        if (c == 0 && r >= kb) {
          const unsigned long long a = abs_key(v);
          if (key_better(a, r, cv, ci)) { cv = a; ci = r; }
        }
      }
      unsigned long long bv;
      int bi;
      block_argmax_key(cv, ci, S.red, &bv, &bi);  // ends with a block barrier: Sp0 is complete
      if (threadIdx.x == 0) {
        g.cand_v[lb] = bv;
        g.cand_i[lb] = bi;
      }
      if (bi >= r_lo && bi < r_hi && threadIdx.x < jb)
        g.cand_row[(int64_t)lb * kGridPanel + threadIdx.x] = Sp0[(bi - r_lo) * kSpStride + threadIdx.x];
      if (kb >= r_lo && kb < r_hi && threadIdx.x < jb) g.row_k[threadIdx.x] = Sp0[(kb - r_lo) * kSpStride + threadIdx.x];
    }
    bounded_barrier(bar, gn, w.err, ep);
    // The elimination of a column but its look-ahead column is deferred to
    // the next step, where warps 1 .. 7 finish it while warp 0 finds the next
    // pivot; its operands are kept in registers (lane = column).
    bool dpend = false;
    double d_prow = 0.0, d_rowk = 0.0, d_rowkc = 0.0, d_inv = 0.0;
    int d_p = 0, d_k = 0, d_c = 0;
    const double* d_in = Sp0;
    double* d_out = Sp1;
    for (int c = 0; c < jb; ++c) {
      const int k = kb + c;
      const int buf = c & 1;
      const double* Sin = buf ? Sp1 : Sp0;
      double* Sout = buf ? Sp0 : Sp1;
      const unsigned long long* cvv = g.cand_v + buf * kMaxGrid;
      const int* cii = g.cand_i + buf * kMaxGrid;
      // warp 0: the pivot (the largest candidate, smallest row on ties: a
      // warp argmax over the group's candidates, the same in every lane),
      // the winner's row, the reciprocal of the pivot (the same division in
      // every lane) and the scaled pivot row; warp 1: the row of position k;
      // warps 1 .. 7: the previous column's deferred elimination. One block
      // barrier publishes them.
      if (threadIdx.x < 32) {
        const int t = threadIdx.x;
        unsigned long long pv = 0;
        int p = 0x7fffffff;
        for (int q = t; q < G; q += 32)
          if (key_better(cvv[q], cii[q], pv, p)) {
            pv = cvv[q];
            p = cii[q];
          }
        for (int o = 16; o; o >>= 1) {
          const unsigned long long ov = __shfl_xor_sync(0xffffffffu, pv, o);
          const int oi = __shfl_xor_sync(0xffffffffu, p, o);
          if (key_better(ov, oi, pv, p)) {
            pv = ov;
            p = oi;
          }
        }
        const bool ok = !(pv == 0 || pv >= 0x7FF0000000000000ull || p < k || p >= n);  // zero, Inf or NaN
        const double rp =
            (ok && t < jb) ? g.cand_row[((int64_t)buf * kMaxGrid + p / rows_per) * kGridPanel + t] : 0.0;
        const double pivot = __shfl_sync(0xffffffffu, rp, c);
        const double rinv = 1.0 / pivot;
        if (t < jb) S.prow[t] = (t == c) ? rinv : rp * rinv;
        if (t == 0) {
          S.bc[0] = rinv;
          S.pivot_row = ok ? p : -1;
        }
        if (glead && ok) {
          g.pivval[k] = pivot;
          g.piv[k] = p;
        }
      } else {
        if (threadIdx.x < 64) {
          const int t = threadIdx.x - 32;
          if (t < jb) S.rowk[t] = g.row_k[buf * kGridPanel + t];
        }
        if (dpend) {
          const int lane = threadIdx.x & 31;
          if (lane < jb && lane != d_c + 1)
            for (int rr = (threadIdx.x >> 5) - 1; rr < my_rows; rr += kWarps - 1) {
              const int r = r_lo + rr;
              double v;
              if (r == d_k) {
                v = d_prow;
              } else {
                const double srcv = (r == d_p) ? d_rowk : d_in[rr * kSpStride + lane];
                const double f = (r == d_p) ? d_rowkc : d_in[rr * kSpStride + d_c];
                v = (lane == d_c) ? -f * d_inv : fma(-f, d_prow, srcv);
              }
              d_out[rr * kSpStride + lane] = v;
            }
        }
      }
      __syncthreads();
      const int p = S.pivot_row;
      if (p < 0) return 1;
      const double inv = S.bc[0];
      // One element of the elimination: row rr (global r) of the block, column cc.
      auto elim = [&](int rr, int r, int cc) -> double {
        if (r == k) return S.prow[cc];
        const double srcv = (r == p) ? S.rowk[cc] : Sin[rr * kSpStride + cc];
        const double f = (r == p) ? S.rowk[c] : Sin[rr * kSpStride + c];
        return (cc == c) ? -f * inv : fma(-f, S.prow[cc], srcv);
      };
      const int c1 = c + 1;
      if (c1 < jb) {
        // look-ahead: column c + 1 of every row first (lane = row), its
        // candidate, then the candidate's full row and the row of position
        // k + 1, published; the block arrives at the group barrier, and the
        // rest of this column's elimination waits for the next step
        unsigned long long cv = 0;
        int ci = 0x7fffffff;
        for (int rr = threadIdx.x; rr < my_rows; rr += kThreads) {
          const int r = r_lo + rr;
          const double val = elim(rr, r, c1);
          Sout[rr * kSpStride + c1] = val;
          if (r > k) {
            const unsigned long long a = abs_key(val);
            if (key_better(a, r, cv, ci)) {
              cv = a;
              ci = r;
            }
          }
        }
        unsigned long long bv;
        int bi;
        block_argmax_key(cv, ci, S.red, &bv, &bi);
        const int nb = c1 & 1;
        if (threadIdx.x == 0) {
          g.cand_v[nb * kMaxGrid + lb] = bv;
          g.cand_i[nb * kMaxGrid + lb] = bi;
        }
        if (threadIdx.x < 32) {
          if (bi >= r_lo && bi < r_hi && threadIdx.x < jb)
            g.cand_row[((int64_t)nb * kMaxGrid + lb) * kGridPanel + threadIdx.x] = elim(bi - r_lo, bi, threadIdx.x);
        } else if (threadIdx.x < 64) {
          const int t = threadIdx.x - 32;
          if (k + 1 >= r_lo && k + 1 < r_hi && t < jb) g.row_k[nb * kGridPanel + t] = elim(k + 1 - r_lo, k + 1, t);
        }
        barrier_arrive(bar, gn, w.err, ep);
        const int lane = threadIdx.x & 31;
        d_prow = lane < jb ? S.prow[lane] : 0.0;
        d_rowk = lane < jb ? S.rowk[lane] : 0.0;
        d_rowkc = S.rowk[c];
        d_inv = inv;
        d_p = p;
        d_k = k;
        d_c = c;
        d_in = Sin;
        d_out = Sout;
        dpend = true;
        barrier_wait(bar, gn, w.err, ep);
      } else {
        // the panel's last column: its whole elimination now (warp w: rows
        // w, w + 8, ...; lane = column)
        const int lane = threadIdx.x & 31;
        if (lane < jb)
          for (int rr = threadIdx.x >> 5; rr < my_rows; rr += kWarps)
            Sout[rr * kSpStride + lane] = elim(rr, r_lo + rr, lane);
        dpend = false;
        bounded_barrier(bar, gn, w.err, ep);
      }
    }
    return 0;
  }

  // The panel's update on the FP64 pipe: panel -> W and its column-major copy
  // Pf, the panel's row swaps on the other columns, pivot rows -> R, then
  // W[:, not J] += (Pf - I_J) R in DMMA tiles.
  __device__ __noinline__ void update_rank32(GjGroup& g, const GjCtx& x, double* W, int n, int kb, int jb) {
    const double* Sf = (jb & 1) ? x.Sp1 : x.Sp0;
    double* Pf = g.panel;
    for (int e = threadIdx.x; e < x.my_rows * jb; e += kThreads) {
      const int rr = e / jb, c = e % jb;
      const int r = x.r_lo + rr;
      const double v = Sf[rr * kSpStride + c];
      W[(int64_t)r * n + kb + c] = v;
      Pf[(int64_t)c * n + r] = v;
    }
    for (int j = x.gt; j < n; j += x.gnt) {
      if (j >= kb && j < kb + jb) continue;
      for (int c = 0; c < jb; ++c) {
        const int k = kb + c, p = g.piv[k];
        if (p != k) {
          const double t0 = W[(int64_t)k * n + j];
          W[(int64_t)k * n + j] = W[(int64_t)p * n + j];
          W[(int64_t)p * n + j] = t0;
        }
      }
      for (int c = 0; c < jb; ++c) g.R[(int64_t)c * n + j] = W[(int64_t)(kb + c) * n + j];
    }
    bounded_barrier(x.bar, x.G, w.err, x.ep);
    const int tiles = (n + kTileM - 1) / kTileM;
    for (int t = x.lb; t < tiles * tiles; t += x.G)
      rank_update_tile(W, n, kb, jb, Pf, g.R, (t / tiles) * kTileM, (t % tiles) * kTileN);
    bounded_barrier(x.bar, x.G, w.err, x.ep);
  }

  // One tensor-core update of W on this block's share of the tiles ut names
  // (skipped once the grid's error word is set).
  __device__ void group_update(GjGroup& g, const GjCtx& x, double* W, int n, const UpdTiles& ut) {
    if (threadIdx.x == 0) S.skip_upd = *(volatile int*)w.err;
    __syncthreads();
    if (S.skip_upd) return;
    const int T = ((n + kUpdM - 1) / kUpdM) * ut.ncbt;
    const int t_lo = (int)((int64_t)x.lb * T / x.G), t_hi = (int)((int64_t)(x.lb + 1) * T / x.G);
    sliced_update(S.slc, reinterpret_cast<unsigned char*>(grid_panel_smem), &maps->a[g.gi], &maps->b[g.gi], g.sl,
                  W, n, ut, t_lo, t_hi, w.err);
  }

  // Rows of U_0 .. U_{q-1} (columns [0, 32 q) of g.ucat) permuted by the row
  // swaps of the sub-panel at kb: each position the swaps touch (J and the
  // pivot rows) gets the row the swaps moved there, traced back through them.
  // One block; all reads before any write.
  __device__ __noinline__ void permute_ucat(GjGroup& g, int kb, int jb, int q) {
    const int np = 2 * jb, cols = q * kGridPanel;
    if ((int)threadIdx.x < np) {
      const int idx = threadIdx.x;
      const int pos = idx < jb ? kb + idx : g.piv[kb + idx - jb];
      int s = pos;
      for (int t = jb - 1; t >= 0; --t) {
        const int k = kb + t, p = g.piv[k];
        s = s == k ? p : (s == p ? k : s);
      }
      S.ppos[idx] = pos;
      S.psrc[idx] = s;
    }
    __syncthreads();
    constexpr int kPer = (2 * kGridPanel * (kSuperCols - kGridPanel) + kThreads - 1) / kThreads;
    const int E = np * cols;
    double buf[kPer];
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
      const int e = threadIdx.x + it * kThreads;
      if (e < E) buf[it] = g.ucat[(int64_t)S.psrc[e / cols] * kSuperCols + e % cols];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
      const int e = threadIdx.x + it * kThreads;
      if (e < E) g.ucat[(int64_t)S.ppos[e / cols] * kSuperCols + e % cols] = buf[it];
    }
    __syncthreads();
  }

  // Gauss-Jordan inversion with the updates on the tensor cores, blocked in
  // super-panels of up to kMaxChunks sub-panels (kSuperCols columns).
  // Within a super-panel each sub-panel q (columns J_q) is factored on the
  // current W[:, J_q] as in the unblocked form, and its rank-32 update reaches
  // at once only the super-panel's other columns (a narrow update). For the
  // columns outside the super-panel the update is deferred: the sub-panel's
  // row swaps are applied to them at once, and its factor U_q = P_q - I_{J_q}
  // (rows permuted by the later sub-panels' swaps) and its pivot rows
  //   v_q = W[J_q, :] + sum_{p < q} U_p[J_q, :] v_p
  // (W swapped but not yet updated there: v_q is the block of pivot rows the
  // unblocked form would meet) are kept in g.ucat and g.vcat. The super-panel
  // ends with one update W[:, outside] += [U_0 .. U_{m-1}] [v_0; ..; v_{m-1}],
  // K = 32 m exact digit products per element, so W is read and written once
  // per super-panel instead of once per panel. Returns 1 for a bad pivot.
  __device__ __noinline__ int gj_blocked(GjGroup& g, const GjCtx& x, double* W, int n) {
    const int lane = threadIdx.x & 31, i8 = lane & 7;
    const int gw = x.gt >> 5, nw = x.gnt >> 5;
    const int ncb = (n + kUpdN - 1) / kUpdN;
    double* UsT = grid_panel_smem + 2 * x.rows_per * kSpStride;  // [32 q][32]: rows J_q of U_0 .. U_{q-1}, transposed
    for (int K0 = 0; K0 < n; K0 += kSuperCols) {
      const int B = min(kSuperCols, n - K0);
      const int m = (B + kGridPanel - 1) / kGridPanel;
      for (int q = 0; q < m; ++q) {
        const int kb = K0 + q * kGridPanel, jb = min(kGridPanel, n - kb);
        if (panel_steps(g, x, W, n, kb, jb)) return 1;
        const double* Sf = (jb & 1) ? x.Sp1 : x.Sp0;
        for (int e = threadIdx.x; e < x.my_rows * jb; e += kThreads) {
          const int rr = e / jb, c = e % jb;
          W[(int64_t)(x.r_lo + rr) * n + kb + c] = Sf[rr * kSpStride + c];
        }
        // U_q = P_q - I_{J_q}, this block's rows, eight lanes per row: FP64
        // into block q of g.ucat, and its digits (one chunk) for the narrow update
        for (int r4 = (threadIdx.x >> 5) * 4; r4 < x.my_rows; r4 += kThreads / 8) {
          const int rr = r4 + (lane >> 3), r = x.r_lo + rr;
          const bool valid = rr < x.my_rows;
          double u[4];
          for (int t = 0; t < 4; ++t) {
            const int c = 4 * i8 + t;
            u[t] = (valid && c < jb) ? Sf[rr * kSpStride + c] - (r == kb + c ? 1.0 : 0.0) : 0.0;
          }
          if (valid) {
            double* up = g.ucat + (int64_t)r * kSuperCols + q * kGridPanel + 4 * i8;
            *reinterpret_cast<double2*>(up) = make_double2(u[0], u[1]);
            *reinterpret_cast<double2*>(up + 2) = make_double2(u[2], u[3]);
          }
          if (m > 1)
            slice_row8_1(u[0], u[1], u[2], u[3], i8, valid, g.sl.adig + (int64_t)r * kDigRow, g.sl.aexp + r);
        }
        // the sub-panel's row swaps as one permutation of the rows they
        // touch: position S.ppos[e] receives the row that was at S.psrc[e]
        // (traced back through the swaps; e < jb: the positions J_q in order,
        // then the pivot rows)
        if ((int)threadIdx.x < 2 * jb) {
          const int idx = threadIdx.x;
          const int pos = idx < jb ? kb + idx : g.piv[kb + idx - jb];
          int s = pos;
          for (int t = jb - 1; t >= 0; --t) {
            const int k = kb + t, p = g.piv[k];
            s = s == k ? p : (s == p ? k : s);
          }
          S.ppos[idx] = pos;
          S.psrc[idx] = s;
        }
        __syncthreads();
        // rows J_q of U_0 .. U_{q-1} as this sub-panel's swaps leave them,
        // transposed into shared memory (UsT[32 p + c2][c] = U_p[kb + c, c2])
        if (q > 0) {
          for (int e = threadIdx.x; e < q * kGridPanel * kGridPanel; e += kThreads) {
            const int c = e % kGridPanel, kq = e / kGridPanel;
            UsT[e] = c < jb ? g.ucat[(int64_t)S.psrc[c] * kSuperCols + kq] : 0.0;
          }
          __syncthreads();
        }
        // every column outside J_q, eight lanes per column (warps walk the
        // columns four at a time, every block of the group taking part): the
        // lanes apply the swaps' permutation to the column (all loads, then
        // all stores; lane i8 holds positions 4 i8 .. + 3 of J_q, the new
        // pivot rows W[J_q, j], and of the pivot rows); then, inside the
        // super-panel, they split W[J_q, j] into digits for the narrow update;
        // outside it they form v_q[:, j] (rows 4 i8 .. 4 i8 + 3) into g.vcat
        for (int j4 = gw * 4; j4 < n; j4 += nw * 4) {
          const int j = j4 + (lane >> 3);
          const bool valid = j < n && (j < kb || j >= kb + jb);
          const bool inside = j >= K0 && j < K0 + B;
          double v[4], pr[4];
          for (int t = 0; t < 4; ++t) {
            const int e = 4 * i8 + t;
            v[t] = (valid && e < jb) ? W[(int64_t)S.psrc[e] * n + j] : 0.0;
            pr[t] = (valid && e < jb) ? W[(int64_t)S.psrc[jb + e] * n + j] : 0.0;
          }
          __syncwarp();  // every load of the column before any store
          if (valid)
            for (int t = 0; t < 4; ++t) {
              const int e = 4 * i8 + t;
              if (e < jb && S.psrc[e] != S.ppos[e]) W[(int64_t)S.ppos[e] * n + j] = v[t];
              if (e < jb && S.psrc[jb + e] != S.ppos[jb + e]) W[(int64_t)S.ppos[jb + e] * n + j] = pr[t];
            }
          if (m > 1)
            slice_row8_1(v[0], v[1], v[2], v[3], i8, valid && inside, g.sl.bdig + (int64_t)j * kDigRow,
                         g.sl.bexp + j);
          const bool outside = valid && !inside;
          double* vc = g.vcat + (int64_t)(outside ? j : 0) * kSuperCols;
          for (int p = 0; p < q; ++p) {
            double a[4] = {0.0, 0.0, 0.0, 0.0};
            if (outside) {
              const double2 a01 = *reinterpret_cast<const double2*>(vc + p * kGridPanel + 4 * i8);
              const double2 a23 = *reinterpret_cast<const double2*>(vc + p * kGridPanel + 4 * i8 + 2);
              a[0] = a01.x;
              a[1] = a01.y;
              a[2] = a23.x;
              a[3] = a23.y;
            }
#pragma unroll
            for (int c2 = 0; c2 < kGridPanel; ++c2) {
              const double b = __shfl_sync(0xffffffffu, a[c2 & 3], (lane & ~7) | (c2 >> 2));
              const double* us = UsT + (p * kGridPanel + c2) * kGridPanel + 4 * i8;
              const double2 u01 = *reinterpret_cast<const double2*>(us);
              const double2 u23 = *reinterpret_cast<const double2*>(us + 2);
              v[0] = fma(u01.x, b, v[0]);
              v[1] = fma(u01.y, b, v[1]);
              v[2] = fma(u23.x, b, v[2]);
              v[3] = fma(u23.y, b, v[3]);
            }
          }
          if (outside) {
            *reinterpret_cast<double2*>(vc + q * kGridPanel + 4 * i8) = make_double2(v[0], v[1]);
            *reinterpret_cast<double2*>(vc + q * kGridPanel + 4 * i8 + 2) = make_double2(v[2], v[3]);
          }
          __syncwarp();
        }
        fence_proxy_async_global();  // the digits are read by TMA after the barrier
        bounded_barrier(x.bar, x.G, w.err, x.ep);
        // the narrow update (block 0 first applies the swaps to U_0 .. U_{q-1})
        if (q > 0 && x.lb == 0) permute_ucat(g, kb, jb, q);
        if (m > 1) {
          const int cb0 = K0 / kUpdN;
          const UpdTiles ut{1, cb0, min(ncb - cb0, (B + kUpdN - 1) / kUpdN), 1 << 30, 0, kb, jb};
          group_update(g, x, W, n, ut);
        }
        bounded_barrier(x.bar, x.G, w.err, x.ep);
      }
      // digits of the deferred update, K = 32 m: every row of
      // [U_0 .. U_{m-1}] and every column of [v_0; ..; v_{m-1}] outside the
      // super-panel, eight lanes per row or column
      const int items = 2 * n - B;
      for (int q4 = gw * 4; q4 < items; q4 += nw * 4) {
        const int it = q4 + (lane >> 3);
        const bool valid = it < items, isa = it < n;
        int row = isa ? it : it - n;
        if (!isa && row >= K0) row += B;
        if (!valid) row = 0;
        const double* sp = (isa ? g.ucat : g.vcat) + (int64_t)row * kSuperCols + 4 * i8;
        double v[4 * kMaxChunks];
#pragma unroll
        for (int c = 0; c < kMaxChunks; ++c) {
          double2 a01 = make_double2(0.0, 0.0), a23 = make_double2(0.0, 0.0);
          if (valid && c < m) {
            a01 = *reinterpret_cast<const double2*>(sp + c * kGridPanel);
            a23 = *reinterpret_cast<const double2*>(sp + c * kGridPanel + 2);
          }
          v[4 * c] = a01.x;
          v[4 * c + 1] = a01.y;
          v[4 * c + 2] = a23.x;
          v[4 * c + 3] = a23.y;
        }
        slice_row8<kMaxChunks>(v, i8, valid, m, (isa ? g.sl.adig : g.sl.bdig) + (int64_t)row * kDigRow,
                               (isa ? g.sl.aexp : g.sl.bexp) + row);
      }
      fence_proxy_async_global();
      bounded_barrier(x.bar, x.G, w.err, x.ep);
      {
        const int cin0 = K0 / kUpdN, cin1 = min(ncb, (K0 + B + kUpdN - 1) / kUpdN);
        const UpdTiles ut{m, 0, ncb - (cin1 - cin0), cin0, cin1 - cin0, K0, B};
        if (ut.ncbt > 0) group_update(g, x, W, n, ut);
      }
      bounded_barrier(x.bar, x.G, w.err, x.ep);
    }
    return 0;
  }

  __device__ void inverse_group(GjGroup& g, int g0, int gn, unsigned long long* bar, unsigned long long* ep,
                                const double* src, double* dst, int n) {
    GjCtx x;
    x.lb = blockIdx.x - g0;
    x.gt = x.lb * kThreads + threadIdx.x;
    x.gnt = gn * kThreads;
    x.G = gn;
    x.rows_per = (n + gn - 1) / gn;
    x.r_lo = x.lb * x.rows_per;
    x.r_hi = min(n, x.r_lo + x.rows_per);
    x.my_rows = x.r_hi > x.r_lo ? x.r_hi - x.r_lo : 0;
    x.Sp0 = grid_panel_smem;                             // [rows_per][kSpStride]
    x.Sp1 = grid_panel_smem + x.rows_per * kSpStride;
    x.bar = bar;
    x.ep = ep;
    const int lb = x.lb, gt = x.gt, gnt = x.gnt, G = x.G;
    const bool glead = lb == 0 && threadIdx.x == 0;
    double* W = g.work;
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = gt; t < nn; t += gnt) W[t] = src[t];
    double ld = 0.0;  // group leader
    int status = 0;
    bounded_barrier(bar, gn, w.err, ep);
    if (maps) {
      status = gj_blocked(g, x, W, n);
    } else {
      for (int kb = 0; kb < n && !status; kb += kGridPanel) {
        const int jb = min(kGridPanel, n - kb);
        status = panel_steps(g, x, W, n, kb, jb);
        if (!status) update_rank32(g, x, W, n, kb, jb);
      }
    }
    if (!status) {
      // log|det| = sum of log|pivot|, one log per thread, per-block partial sums
      double lsum = 0.0;
      for (int k = gt; k < n; k += gnt) lsum += log(fabs(g.pivval[k]));
      lsum = block_sum(lsum, S.red);
      if (threadIdx.x == 0) g.ldpart[lb] = lsum;
      if (glead) {
        for (int j = 0; j < n; ++j) g.perm[j] = j;
        for (int k = n - 1; k >= 0; --k) {
          const int p = g.piv[k];
          const int t0 = g.perm[k];
          g.perm[k] = g.perm[p];
          g.perm[p] = t0;
        }
      }
      bounded_barrier(bar, gn, w.err, ep);
      if (glead)
        for (int q = 0; q < G; ++q) ld += g.ldpart[q];
      for (int64_t t = gt; t < nn; t += gnt) {
        const int64_t i = t / n, j = t % n;
        dst[t] = W[i * n + g.perm[j]];
      }
    }
    if (glead) {
      g.result[0] = ld;
      g.result[1] = status;
    }
  }

  // dst <- src^{-1} on the whole grid; returns 0, or 1 for a zero / non-finite pivot.
  __device__ int inverse(const double* src, double* dst, int n, double* logabsdet) {
    inverse_group(w.gj[0], 0, gridDim.x, w.bar, &S.ep[0], src, dst, n);
    sync();
    *logabsdet = w.gj[0].result[0];
    const int st = w.gj[0].result[1] != 0.0;
    sync();
    return st;
  }

  // Xi <- X^{-1} and Yi <- Y^{-1} at the same time, each on one half of the
  // grid (blocks b and b + G/2 share an SM, so one group's panel steps overlap
  // the other group's rank updates on the FP64 pipe).
  __device__ int inverse_pair(const double* X, double* Xi, const double* Y, double* Yi, int n, double* ldx,
                              double* ldy) {
    const int half = gridDim.x / 2;
    if (half < 8) {
      const int a = inverse(X, Xi, n, ldx);
      const int b = inverse(Y, Yi, n, ldy);
      return a | b;
    }
    if ((int)blockIdx.x < half)
      inverse_group(w.gj[0], 0, half, w.gj[0].bar, &S.ep[1], X, Xi, n);
    else
      inverse_group(w.gj[1], half, gridDim.x - half, w.gj[1].bar, &S.ep[2], Y, Yi, n);
    sync();
    *ldx = w.gj[0].result[0];
    *ldy = w.gj[1].result[0];
    const int st = (w.gj[0].result[1] != 0.0) || (w.gj[1].result[1] != 0.0);
    sync();
    return st;
  }

  __device__ void tally_reset() {
    if (threadIdx.x == 0) S.work[0] = S.work[1] = S.work[2] = S.work[3] = 0;
  }
  __device__ void tally(int i, int c) {
    if (threadIdx.x == 0) S.work[i] += c;
  }
  __device__ int tally_get(int i) const { return S.work[i]; }
};

}  // namespace lg
