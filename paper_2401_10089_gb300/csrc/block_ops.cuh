// block_ops.cuh -- the one-thread-block-per-matrix ops layer (n <= kMaxN):
// vectors in shared memory, reductions through shared memory, matrices in the
// block's workspace slot.
#pragma once

#include "cta_linalg.cuh"

namespace LG_NS {

struct BlockOps {
  BlockSmem& S;

  __device__ int tid() const { return threadIdx.x; }
  __device__ int nthreads() const { return kThreads; }
  __device__ void sync() { __syncthreads(); }
  __device__ bool leader() const { return threadIdx.x == 0; }

  __device__ double sum(double v) { return block_sum(v, S.red); }
  __device__ double max(double v) { return block_max(v, S.red); }
  __device__ int all(int v) { return block_and(v, S.red); }
  __device__ void argmax(double v, int i, double* ov, int* oi) { block_argmax(v, i, S.red, ov, oi); }

  // A scalar as thread 0 computed it, for every thread of the block.
  __device__ double bcast0(double v) {
    if (threadIdx.x == 0) S.bc[0] = v;
    __syncthreads();
    const double r = S.bc[0];
    __syncthreads();
    return r;
  }

  __device__ double* vec(int i) {
    return i == 0 ? S.vec.x : (i == 1 ? S.vec.y : (i == 2 ? S.vec.t : S.vec.z));
  }

  __device__ double norm1(const double* M, int n, double shift) { return mat_norm1(M, n, shift, S.red); }

  __device__ void matvec(const double* M, int n, double shift, const double* x, double* y, int trans) {
    mat_vec(M, n, shift, x, y, trans);
  }

  // Denman-Beavers update, eq. (ScalDB): X <- (mu X + Yi / mu) / 2, Y <- (mu Y +
  // Xi / mu) / 2 (one thread per column); returns ||X_new - X_old||_1, ||X_new||_1.
  __device__ void db_update(double* X, double* Y, const double* Xi, const double* Yi, double mu, double imu, int n,
                            double* nd, double* nx) {
    double sd = 0.0, sx = 0.0;
    for (int j = threadIdx.x; j < n; j += kThreads) {
      double cd = 0.0, cx = 0.0;
      for (int i = 0; i < n; ++i) {
        const int64_t q = (int64_t)i * n + j;
        const double xo = X[q];
        const double xn = 0.5 * fma(mu, xo, Yi[q] * imu);
        Y[q] = 0.5 * fma(mu, Y[q], Xi[q] * imu);
        X[q] = xn;
        cd += fabs(xn - xo);
        cx += fabs(xn);
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
    double sd = 0.0, sx = 0.0;
    for (int j = threadIdx.x; j < n; j += kThreads) {
      double cd = 0.0, cx = 0.0;
      for (int i = 0; i < n; ++i) {
        const int64_t q = (int64_t)i * n + j;
        const double xo = X[q];
        const double xmi = first ? (i == j ? 1.0 : 0.0) : XMi[q];
        const double xn = 0.5 * fma(mu, xo, xmi * imu);
        Mk[q] = fma(0.25, fma(mu2, Mk[q], Mi[q] * imu2), i == j ? 0.5 : 0.0);
        X[q] = xn;
        cd += fabs(xn - xo);
        cx += fabs(xn);
      }
      sd = nanmax(sd, cd);
      sx = nanmax(sx, cx);
    }
    *nd = max(sd);
    *nx = max(sx);
  }

  __device__ void gemm(int n, const double* A, double as, const double* B, double bs, double alpha,
                       const EpiTerms& e, OutView out, bool ta = false, bool tb = false) {
    gemm_block(n, A, as, B, bs, alpha, e, out, S.u.gemm, ta, tb);
  }

  __device__ void lincomb(int n, const EpiTerms& e, double* out) { lincomb_block(n, e, out); }

  // dst <- src^{-1}; returns 0, or 1 for a zero / non-finite pivot.
  __device__ int inverse(const double* src, double* dst, int n, double* logabsdet) {
    mat_copy(dst, src, n);
    __syncthreads();
    return gj_inverse_block(dst, n, logabsdet, S);
  }

  // Xi <- X^{-1}, Yi <- Y^{-1} (one after the other on this block).
  __device__ int inverse_pair(const double* X, double* Xi, const double* Y, double* Yi, int n, double* ldx,
                              double* ldy) {
    const int a = inverse(X, Xi, n, ldx);
    if (a) return a;
    return inverse(Y, Yi, n, ldy);
  }

  __device__ void tally_reset() {
    if (threadIdx.x == 0) S.work[0] = S.work[1] = S.work[2] = S.work[3] = 0;
  }
  __device__ void tally(int i, int c) {
    if (threadIdx.x == 0) S.work[i] += c;
  }
  __device__ int tally_get(int i) const { return S.work[i]; }
};

}  // namespace LG_NS
