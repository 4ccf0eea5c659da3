// cta_linalg.cuh -- CTA-level FP64 dense linear algebra for one matrix per
// thread block (n <= kMaxN). Everything here runs on the FP64 pipe, which on
// GB300 is the bottleneck by a wide margin (about 1 TFLOP/s for the chip), so
// the routines keep every FP64 instruction useful: divisions, logarithms and
// exponentials are computed once per CTA and broadcast through shared memory,
// index arithmetic stays in integer registers, and the O(n^3) parts run as
// DMMA (mma.sync m8n8k4 f64) tiles or register-blocked DFMA.
//
// Matrices live in global memory (L2-resident working set), row-major with
// leading dimension n. All block-wide control flow is uniform: every scalar
// that decides a branch comes out of a block reduction broadcast through
// shared memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// One translation unit builds one block configuration: LG_NS names its
// namespace, LG_THREADS the block size, LG_MAXN the largest n, LG_TILE the
// DMMA output tile (64: 8 warps of 16 x 32; 32: warps of 16 x 16 or 16 x 32).
#ifndef LG_NS
#define LG_NS lg
#define LG_THREADS 256
#define LG_MAXN 256
#define LG_TILE 64
#define LG_MINBLOCKS 2
#endif

namespace lg {}
namespace LG_NS {
using namespace ::lg;

constexpr int kThreads = LG_THREADS;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxN = LG_MAXN;  // largest n of this one-block-per-matrix configuration
constexpr int kPanel = 16;      // Gauss-Jordan panel width
constexpr int kTileM = LG_TILE, kTileN = LG_TILE, kTileK = 16;
constexpr int kWarpsM = (LG_TILE == 64) ? 4 : 2;   // warps along the tile's rows
constexpr int kWarpsN = kWarps / kWarpsM;          // warps along its columns
constexpr int kMB = kTileM / kWarpsM / 8;          // 8-row DMMA blocks per warp
constexpr int kNB = kTileN / kWarpsN / 8;          // 8-column DMMA blocks per warp
constexpr int kAsStride = kTileK + 4;  // shared-memory row strides that keep
constexpr int kBsStride = kTileN + 4;  // DMMA fragment loads conflict-free
static_assert(kWarpsM * kWarpsN == kWarps && kMB >= 1 && kNB >= 1, "tile / warp layout");

struct Reduce {
  double v[kWarps];
  int i[kWarps];
};

struct GemmSmem {
  double As[kTileM * kAsStride];
  double Bs[kTileK * kBsStride];
};

struct GjSmem {
  double P[kPanel * kMaxN];  // panel, column-major: P[c * kMaxN + i]
  double R[kPanel * kMaxN];  // rows of the panel's pivots, R[c * kMaxN + j]
};

struct VecSmem {
  double x[kMaxN], y[kMaxN], z[kMaxN], t[kMaxN];
};

struct BlockSmem {
  union {
    GemmSmem gemm;
    GjSmem gj;
  } u;
  VecSmem vec;
  int piv[kMaxN];
  Reduce red;
  double bc[4];  // broadcast slots
  int ibc[4];
  int work[4];   // thread 0's tally: DB iterations, inverses, products, matvecs
};

// ---------------------------------------------------------------------------
// Block reductions (all threads get the result).
// ---------------------------------------------------------------------------
static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

static __device__ __forceinline__ double nanmax(double a, double b) {
  return (a > b || a != a) ? a : b;
}

static __device__ double block_sum(double v, Reduce& r) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) r.v[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < kWarps; ++t) s += r.v[t];
  __syncthreads();
  return s;
}

static __device__ double block_max(double v, Reduce& r) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) r.v[w] = v;
  __syncthreads();
  double s = r.v[0];
#pragma unroll
  for (int t = 1; t < kWarps; ++t) s = nanmax(s, r.v[t]);
  __syncthreads();
  return s;
}

// |v| as an integer whose order is that of |v| (IEEE binary64 magnitudes order
// like their bit patterns); NaN maps to the key of +Inf, so a NaN pivot is
// taken like an infinite one and then rejected. Integer work only: on this
// GPU every FP64 instruction on the pivot search's critical path is costly.
static __device__ __forceinline__ unsigned long long abs_key(double v) {
  unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
  return b > 0x7FF0000000000000ull ? 0x7FF0000000000000ull : b;
}
static __device__ __forceinline__ bool key_better(unsigned long long a, int ia, unsigned long long b, int ib) {
  return a > b || (a == b && ia < ib);
}

// Block argmax over (key, index): largest key, smallest index on ties; the
// result in every thread. Ends with a block barrier.
static __device__ void block_argmax_key(unsigned long long key, int idx, Reduce& r, unsigned long long* ok,
                                        int* oi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (key_better(k2, i2, key, idx)) {
      key = k2;
      idx = i2;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    r.v[w] = __longlong_as_double(static_cast<long long>(key));
    r.i[w] = idx;
  }
  __syncthreads();
  unsigned long long bk = static_cast<unsigned long long>(__double_as_longlong(r.v[0]));
  int bi = r.i[0];
#pragma unroll
  for (int t = 1; t < kWarps; ++t) {
    const unsigned long long kt = static_cast<unsigned long long>(__double_as_longlong(r.v[t]));
    if (key_better(kt, r.i[t], bk, bi)) {
      bk = kt;
      bi = r.i[t];
    }
  }
  __syncthreads();
  *ok = bk;
  *oi = bi;
}

// max of v with the smallest index among ties; v < 0 marks "not a candidate".
static __device__ void block_argmax(double v, int idx, Reduce& r, double* out_v, int* out_i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (v2 > v || (v2 == v && i2 < idx)) {
      v = v2;
      idx = i2;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    r.v[w] = v;
    r.i[w] = idx;
  }
  __syncthreads();
  double bv = r.v[0];
  int bi = r.i[0];
#pragma unroll
  for (int t = 1; t < kWarps; ++t)
    if (r.v[t] > bv || (r.v[t] == bv && r.i[t] < bi)) {
      bv = r.v[t];
      bi = r.i[t];
    }
  __syncthreads();
  *out_v = bv;
  *out_i = bi;
}

static __device__ int block_and(int pred, Reduce& r) {
  int w_all = __all_sync(0xffffffffu, pred);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) r.i[w] = w_all;
  __syncthreads();
  int a = 1;
#pragma unroll
  for (int t = 0; t < kWarps; ++t) a &= r.i[t];
  __syncthreads();
  return a;
}

// ---------------------------------------------------------------------------
// Elementwise helpers over an n x n matrix (ld = n).
// ---------------------------------------------------------------------------
static __device__ void mat_copy(double* __restrict__ dst, const double* __restrict__ src, int n) {
  const int nn = n * n;
  for (int t = threadIdx.x; t < nn; t += kThreads) dst[t] = src[t];
}

static __device__ void mat_identity(double* __restrict__ dst, int n) {
  const int nn = n * n;
  for (int t = threadIdx.x; t < nn; t += kThreads) dst[t] = (t / n == t % n) ? 1.0 : 0.0;
}

// ||M - shift I||_1 = max_j sum_i |m_ij - shift delta_ij|. NaN propagates.
static __device__ double mat_norm1(const double* __restrict__ M, int n, double shift, Reduce& r) {
  double best = 0.0;
  for (int j = threadIdx.x; j < n; j += kThreads) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
      double v = M[i * n + j];
      if (i == j) v -= shift;
      s += fabs(v);
    }
    best = nanmax(best, s);
  }
  return block_max(best, r);
}

// y = (M - shift I) x (trans = 0) or y = (M - shift I)^T x (trans = 1);
// x, y in shared memory (distinct).
static __device__ void mat_vec(const double* __restrict__ M, int n, double shift, const double* x,
                        double* y, int trans) {
  if (!trans) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = w; i < n; i += kWarps) {
      double s = 0.0;
      for (int c = l; c < n; c += 32) s = fma(M[i * n + c], x[c], s);
      s = warp_sum(s);
      if (l == 0) y[i] = s - shift * x[i];
    }
  } else {
    for (int j = threadIdx.x; j < n; j += kThreads) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s = fma(M[i * n + j], x[i], s);
      y[j] = s - shift * x[j];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// GEMM: out = alpha * (A - a_shift I)(B - b_shift I) + sum_t c_t E_t,
// FP64 DMMA (mma.sync.m8n8k4.f64) on 64 x 64 output tiles.
// ---------------------------------------------------------------------------
struct EpiTerms {
  const double* M[6];
  double c[6];
  int count;
};

struct OutView {
  void* p;     // element 0 of the matrix
  int dtype;   // 0: F64, 1: F32
};

static __device__ __forceinline__ void store_out(const OutView& o, size_t idx, double v) {
  if (o.dtype == 0)
    static_cast<double*>(o.p)[idx] = v;
  else
    static_cast<float*>(o.p)[idx] = static_cast<float>(v);
}

static __device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// One 64 x 64 output tile (rows r0.., cols c0..) of
// out = alpha * op(A - a_shift I) op(B - b_shift I) + sum_t c_t E_t, by DMMA
// with the block's 8 warps (each a 16 x 32 sub-tile); op(M) = M^T when the
// transpose flag is set. A, B, E, out: n x n, ld n. `out` may be one of the
// E_t (each element is read before it is written by the same thread).
static __device__ void gemm_tile(int n, int r0, int c0, const double* __restrict__ A, double a_shift,
                          const double* __restrict__ B, double b_shift, double alpha,
                          const EpiTerms& epi, OutView out, GemmSmem& sm, bool ta = false, bool tb = false) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / kWarpsN, wn = warp % kWarpsN;
  const int g = lane >> 2, q = lane & 3;
  constexpr int RW = kTileM / kWarpsM, CW = kTileN / kWarpsN;  // rows, columns of a warp's sub-tile
  double acc[kMB][kNB][2];
#pragma unroll
  for (int a = 0; a < kMB; ++a)
#pragma unroll
    for (int b = 0; b < kNB; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
  for (int k0 = 0; k0 < n; k0 += kTileK) {
#pragma unroll
    for (int e = tid; e < kTileM * kTileK; e += kThreads) {
      const int rr = e / kTileK, kk = e % kTileK;
      const int gr = r0 + rr, gk = k0 + kk;
      double v = 0.0;
      if (gr < n && gk < n) {
        v = ta ? A[(size_t)gk * n + gr] : A[(size_t)gr * n + gk];
        if (gr == gk) v -= a_shift;
      }
      sm.As[rr * kAsStride + kk] = v;
    }
#pragma unroll
    for (int e = tid; e < kTileK * kTileN; e += kThreads) {
      const int kk = e / kTileN, cc = e % kTileN;
      const int gk = k0 + kk, gc = c0 + cc;
      double v = 0.0;
      if (gk < n && gc < n) {
        v = tb ? B[(size_t)gc * n + gk] : B[(size_t)gk * n + gc];
        if (gk == gc) v -= b_shift;
      }
      sm.Bs[kk * kBsStride + cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTileK; ks += 4) {
      double af[kMB], bf[kNB];
#pragma unroll
      for (int mb = 0; mb < kMB; ++mb) af[mb] = sm.As[(wm * RW + mb * 8 + g) * kAsStride + ks + q];
#pragma unroll
      for (int nb = 0; nb < kNB; ++nb) bf[nb] = sm.Bs[(ks + q) * kBsStride + wn * CW + nb * 8 + g];
#pragma unroll
      for (int mb = 0; mb < kMB; ++mb)
#pragma unroll
        for (int nb = 0; nb < kNB; ++nb) dmma_8x8x4(acc[mb][nb][0], acc[mb][nb][1], af[mb], bf[nb]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mb = 0; mb < kMB; ++mb)
#pragma unroll
    for (int nb = 0; nb < kNB; ++nb)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gr = r0 + wm * RW + mb * 8 + g;
        const int gc = c0 + wn * CW + nb * 8 + 2 * q + h;
        if (gr < n && gc < n) {
          const size_t idx = (size_t)gr * n + gc;
          double v = alpha * acc[mb][nb][h];
          for (int t = 0; t < epi.count; ++t) v = fma(epi.c[t], epi.M[t][idx], v);
          store_out(out, idx, v);
        }
      }
}

static __device__ void gemm_block(int n, const double* __restrict__ A, double a_shift,
                           const double* __restrict__ B, double b_shift, double alpha,
                           const EpiTerms& epi, OutView out, GemmSmem& sm, bool ta = false, bool tb = false) {
  const int tiles = (n + kTileM - 1) / kTileM;
  for (int tile = 0; tile < tiles * tiles; ++tile)
    gemm_tile(n, (tile / tiles) * kTileM, (tile % tiles) * kTileN, A, a_shift, B, b_shift, alpha, epi, out, sm,
              ta, tb);
  __syncthreads();
}

// out = sum_t c_t E_t elementwise (lin-comb node of the computation graph).
static __device__ void lincomb_block(int n, const EpiTerms& e, double* __restrict__ out) {
  const int nn = n * n;
  for (int t = threadIdx.x; t < nn; t += kThreads) {
    double v = 0.0;
    for (int s = 0; s < e.count; ++s) v = fma(e.c[s], e.M[s][t], v);
    out[t] = v;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// In-place inverse by blocked Gauss-Jordan elimination with partial pivoting
// (the left division X \ I of the square-root iteration). Each step k picks
// the largest |w_ik|, i >= k, swaps rows k and p, scales row k by 1/w_kk and
// eliminates column k from every other row; the eliminated column is replaced
// by the column of the elementary transform, so that after the n steps and
// the reverse column swaps W holds A^{-1}. Panels of kPanel columns are
// factorised in shared memory; the rest of W gets the rank-kPanel update
// W[:, notJ] += (M_J - I)[:, J] W[J, notJ] once per panel.
// Returns 0, or 1 if a pivot is zero or not finite. *logabsdet (thread 0
// accumulates; broadcast at the end) = sum log|pivot| = log|det A|.
// ---------------------------------------------------------------------------
static __device__ int gj_inverse_block(double* __restrict__ W, int n, double* logabsdet, BlockSmem& S) {
  const int tid = threadIdx.x;
  double* P = S.u.gj.P;
  double* R = S.u.gj.R;
  int* piv = S.piv;
  // |det| as dm * 2^dex (thread 0): one multiply per step instead of a log,
  // dm kept in [1, 2) by moving its exponent into dex (exact)
  double dm = 1.0, ld_slow = 0.0;
  long long dex = 0;
  int status = 0;
  for (int kb = 0; kb < n && !status; kb += kPanel) {
    const int jb = min(kPanel, n - kb);
    // panel -> shared (column-major)
    for (int e = tid; e < jb * n; e += kThreads) {
      const int c = e / n, i = e % n;
      P[c * kMaxN + i] = W[i * n + kb + c];
    }
    __syncthreads();
    for (int c = 0; c < jb; ++c) {
      const int k = kb + c;
      unsigned long long cand = 0;
      int cidx = n;
      for (int i = tid; i < n; i += kThreads) {
        if (i >= k) {
          const unsigned long long v = abs_key(P[c * kMaxN + i]);  // NaN pivots are taken (and rejected below)
          if (key_better(v, i, cand, cidx)) {
            cand = v;
            cidx = i;
          }
        }
      }
      unsigned long long pv;
      int p;
      block_argmax_key(cand, cidx, S.red, &pv, &p);
      if (pv == 0 || pv >= 0x7FF0000000000000ull) {  // zero, Inf or NaN
        status = 1;
        break;
      }
      if (tid < jb && p != k) {
        double t0 = P[tid * kMaxN + k];
        P[tid * kMaxN + k] = P[tid * kMaxN + p];
        P[tid * kMaxN + p] = t0;
      }
      if (tid == 0) piv[k] = p;
      __syncthreads();
      if (tid == 0) {
        const double d = P[c * kMaxN + k];
        S.bc[0] = 1.0 / d;
        const unsigned long long bits =
            static_cast<unsigned long long>(__double_as_longlong(dm * d)) & 0x7FFFFFFFFFFFFFFFull;
        const int ef = (int)(bits >> 52);
        if (ef == 0 || ef == 0x7FF) {  // subnormal or overflow: fall back to a log
          ld_slow += log(fabs(d));
        } else {
          dex += ef - 1023;
          dm = __longlong_as_double(static_cast<long long>((bits & 0x000FFFFFFFFFFFFFull) | (1023ull << 52)));
        }
      }
      __syncthreads();
      const double inv = S.bc[0];
      if (tid < jb) {
        double* pk = &P[tid * kMaxN + k];
        *pk = (tid == c) ? inv : (*pk) * inv;
      }
      __syncthreads();
      for (int i = tid; i < n; i += kThreads) {
        if (i == k) continue;
        const double f = P[c * kMaxN + i];
        if (f == 0.0) continue;
        P[c * kMaxN + i] = 0.0;
        for (int cc = 0; cc < jb; ++cc) P[cc * kMaxN + i] = fma(-f, P[cc * kMaxN + k], P[cc * kMaxN + i]);
      }
      __syncthreads();
    }
    if (status) break;
    // panel -> W, row swaps of the panel on the other columns, copy of the pivot rows
    for (int e = tid; e < jb * n; e += kThreads) {
      const int c = e / n, i = e % n;
      W[i * n + kb + c] = P[c * kMaxN + i];
    }
    for (int j = tid; j < n; j += kThreads) {
      if (j >= kb && j < kb + jb) continue;
      for (int c = 0; c < jb; ++c) {
        const int k = kb + c, p = piv[k];
        if (p != k) {
          double t0 = W[k * n + j];
          W[k * n + j] = W[p * n + j];
          W[p * n + j] = t0;
        }
      }
      for (int c = 0; c < jb; ++c) R[c * kMaxN + j] = W[(kb + c) * n + j];
    }
    __syncthreads();
    // W[:, notJ] += (P - I_J) R, 4 x 4 register blocks
    const int ngrp = (n + 3) / 4;
    for (int blk = tid; blk < ngrp * ngrp; blk += kThreads) {
      const int i0 = (blk / ngrp) * 4, j0 = (blk % ngrp) * 4;
      // (P - I_J) R = P R - R on the rows of J: start those rows from -R.
      double acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = i0 + a;
        const bool inJ = i >= kb && i < kb + jb;
#pragma unroll
        for (int b = 0; b < 4; ++b)
          acc[a][b] = (inJ && j0 + b < n) ? -R[(i - kb) * kMaxN + j0 + b] : 0.0;
      }
      for (int c = 0; c < jb; ++c) {
        double d[4], rr[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int i = i0 + a;
          d[a] = (i < n) ? P[c * kMaxN + i] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) rr[b] = (j0 + b < n) ? R[c * kMaxN + j0 + b] : 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(d[a], rr[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + a, j = j0 + b;
          if (i < n && j < n && (j < kb || j >= kb + jb)) W[i * n + j] += acc[a][b];
        }
    }
    __syncthreads();
  }
  if (!status) {
    // undo the pivoting on the columns, last step first
    for (int i = tid; i < n; i += kThreads)
      for (int k = n - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k) {
          double t0 = W[i * n + k];
          W[i * n + k] = W[i * n + p];
          W[i * n + p] = t0;
        }
      }
  }
  if (tid == 0) S.bc[1] = log(dm) + (double)dex * 0.69314718055994530942 + ld_slow;
  __syncthreads();
  *logabsdet = S.bc[1];
  __syncthreads();
  return status;
}

}  // namespace LG_NS
