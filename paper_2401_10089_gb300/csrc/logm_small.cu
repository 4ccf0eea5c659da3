// logm_small.cu -- Algorithm 1 of arXiv 2401.10089 (Sec. 6) with one thread
// block per matrix, for n <= kMaxN. A persistent grid pulls matrices from a
// device work queue, so a ragged batch of thousands of matrices is one launch
// and every data-dependent loop (square-root count s, Denman-Beavers
// iterations, estimator sweeps) runs on the device with no host round trip.
//
// Per block, the working matrices live in a workspace slot of kSlotMats
// n_max x n_max FP64 buffers (L2-resident):
//   Acur  current A (the Denman-Beavers X in place), later P_2 = X = I - A
//   A2    saved A_2, then A_I2 = A_2 - 2A + I (eq. AI2) = P_3
//   Y     Denman-Beavers Y, later P_4
//   W1,W2 inverses of X and Y, later P_5, P_6
//   T1,T2 lin-comb nodes (the two factors of the next product)
#include <cmath>
#include <cstdio>

#include "cta_linalg.cuh"
#include "logm_internal.h"

namespace lg {

// Table table_simple_experiment (Sec. 3): the k = 5 scheme fitted to
// -log(1 - x). h_{j,i}, g_{j,i} for j = 2..5, i = 2..j+1 in that order.
__constant__ double c_h5[14] = {
    7.363757032799957e-02, -1.050281301619960e+00, 8.897468955192446e-02,
    -1.599651928992725e-01, 9.577281350989334e-01, 5.394999133948797e-01,
    6.700731102561937e-02, -5.158769100223212e-02, 1.094308587350110e+00,
    1.027072285939197e-01, -8.964023050065877e-03, -2.100705663612491e-01,
    1.949655359168707e-01, 1.117368056772713e+00};
__constant__ double c_g5[14] = {
    -9.666134174379001e-01, -4.395519034717933e-01, 1.048664069004776e-01,
    1.585606124033259e-01, 1.668066506920988e-01, -8.025600931705978e-02,
    -1.159854366397558e-01, 1.066554944706011e-01, 1.127094008297975e+00,
    2.702180425508705e-01, 4.137541209720699e-02, 4.857347452405025e-01,
    -6.000256005636980e-01, 1.063393233943084e+00};
// y_1 .. y_7 (y_1 = 0: no identity term)
__constant__ double c_y5[7] = {0.0, 1.0, 5.065546620208965e-01, 3.832512052972577e-01,
                               1.088307723749078e+00, 2.787461897212877e-01,
                               8.157421998489228e-01};

constexpr double kUnitRoundoff = 0x1p-53;

struct Slot {
  double *Acur, *A2, *Y, *W1, *W2, *T1, *T2;
};

__device__ __forceinline__ int m_of_k(int k) { return k == 1 ? 2 : (k == 2 ? 4 : 14); }
__device__ __forceinline__ int theta_slot(int k) { return k == 1 ? 0 : (k == 2 ? 1 : 2); }

// x^m by repeated multiplication, so that "x^{1/m} <= Theta" is decided as
// "x <= Theta^m" exactly the same way in every implementation.
__device__ __forceinline__ double ipow(double x, int m) {
  double r = 1.0;
  for (int i = 0; i < m; ++i) r *= x;
  return r;
}

__device__ __forceinline__ double load_elem(const void* base, int dtype, int64_t idx) {
  return dtype == 0 ? static_cast<const double*>(base)[idx]
                    : static_cast<double>(static_cast<const float*>(base)[idx]);
}

// dst (F64, ld n) <- src (caller layout); returns 1 if every entry is finite.
__device__ int load_matrix(const void* src, int dtype, int64_t off, int n, double* dst, Reduce& r) {
  int ok = 1;
  const int nn = n * n;
  for (int t = threadIdx.x; t < nn; t += kThreads) {
    const double v = load_elem(src, dtype, off + t);
    ok &= isfinite(v) ? 1 : 0;
    dst[t] = v;
  }
  return block_and(ok, r);
}

__device__ void store_matrix(void* dst, int dtype, int64_t off, int n, const double* src) {
  const int nn = n * n;
  OutView o{dtype == 0 ? static_cast<void*>(static_cast<double*>(dst) + off)
                       : static_cast<void*>(static_cast<float*>(dst) + off),
            dtype};
  for (int t = threadIdx.x; t < nn; t += kThreads) store_out(o, t, src[t]);
}

__device__ void fill_nan(void* dst, int dtype, int64_t off, int n) {
  const int nn = n * n;
  OutView o{dtype == 0 ? static_cast<void*>(static_cast<double*>(dst) + off)
                       : static_cast<void*>(static_cast<float*>(dst) + off),
            dtype};
  for (int t = threadIdx.x; t < nn; t += kThreads) store_out(o, t, __longlong_as_double(0x7ff8000000000000ll));
}

__device__ OutView out_view(void* base, int dtype, int64_t off) {
  return OutView{dtype == 0 ? static_cast<void*>(static_cast<double*>(base) + off)
                            : static_cast<void*>(static_cast<float*>(base) + off),
                 dtype};
}

// ---------------------------------------------------------------------------
// 1-norm estimate of ||B^p||_1, B = Acur - I (Higham 1988, the estimator the
// paper cites in Sec. 6). With A_I2 = B^2 (eq. AI2) the power is applied as
// B^{p mod 2} A_I2^{p div 2} (Sec. 6, item 2). One vector, at most 5 sweeps,
// ties to the smallest index, sign(0) = +1, then the alternating-sign test.
// ---------------------------------------------------------------------------

// v <- M v (trans = 0) or M^T v (trans = 1), M = B^q A_I2^r; tmp is scratch.
__device__ void apply_power(const double* Acur, const double* AI2, int n, int p, double* v,
                            double* tmp, int trans, int* work) {
  const int q = AI2 ? (p & 1) : p;
  const int r = AI2 ? (p >> 1) : 0;
  double* cur = v;
  double* oth = tmp;
  if (threadIdx.x == 0) work[3] += q + r;
  if (!trans) {
    for (int t = 0; t < r; ++t) {
      mat_vec(AI2, n, 0.0, cur, oth, 0);
      double* s = cur; cur = oth; oth = s;
    }
    for (int t = 0; t < q; ++t) {
      mat_vec(Acur, n, 1.0, cur, oth, 0);
      double* s = cur; cur = oth; oth = s;
    }
  } else {
    for (int t = 0; t < q; ++t) {
      mat_vec(Acur, n, 1.0, cur, oth, 1);
      double* s = cur; cur = oth; oth = s;
    }
    for (int t = 0; t < r; ++t) {
      mat_vec(AI2, n, 0.0, cur, oth, 1);
      double* s = cur; cur = oth; oth = s;
    }
  }
  if (cur != v) {
    for (int i = threadIdx.x; i < n; i += kThreads) v[i] = cur[i];
    __syncthreads();
  }
}

__device__ double vec_abs_sum(const double* v, int n, Reduce& r) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) s += fabs(v[i]);
  return block_sum(s, r);
}

__device__ double normest_pow(const double* Acur, const double* AI2, int n, int p, BlockSmem& S) {
  double* x = S.vec.x;
  double* tmp = S.vec.y;
  double* xi = S.vec.t;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += kThreads) x[i] = 1.0 / n;
  __syncthreads();
  apply_power(Acur, AI2, n, p, x, tmp, 0, S.work);
  double est = vec_abs_sum(x, n, S.red);
  if (n > 1) {
    for (int i = tid; i < n; i += kThreads) {
      xi[i] = (x[i] >= 0.0) ? 1.0 : -1.0;
      x[i] = xi[i];
    }
    __syncthreads();
    apply_power(Acur, AI2, n, p, x, tmp, 1, S.work);
    double bv;
    int j;
    {
      double cv = -1.0;
      int ci = n;
      for (int i = tid; i < n; i += kThreads) {
        const double a = fabs(x[i]);
        if (a > cv) { cv = a; ci = i; }
      }
      block_argmax(cv, ci, S.red, &bv, &j);
    }
    for (int sweep = 2; sweep <= 5; ++sweep) {
      for (int i = tid; i < n; i += kThreads) x[i] = (i == j) ? 1.0 : 0.0;
      __syncthreads();
      apply_power(Acur, AI2, n, p, x, tmp, 0, S.work);
      const double est_new = vec_abs_sum(x, n, S.red);
      int same = 1;
      for (int i = tid; i < n; i += kThreads) same &= (((x[i] >= 0.0) ? 1.0 : -1.0) == xi[i]);
      same = block_and(same, S.red);
      if (same || est_new <= est) {
        if (est_new > est) est = est_new;
        break;
      }
      est = est_new;
      for (int i = tid; i < n; i += kThreads) {
        xi[i] = (x[i] >= 0.0) ? 1.0 : -1.0;
        x[i] = xi[i];
      }
      __syncthreads();
      apply_power(Acur, AI2, n, p, x, tmp, 1, S.work);
      const int jlast = j;
      double cv = -1.0;
      int ci = n;
      for (int i = tid; i < n; i += kThreads) {
        const double a = fabs(x[i]);
        if (a > cv) { cv = a; ci = i; }
      }
      block_argmax(cv, ci, S.red, &bv, &j);
      const double zlast = fabs(x[jlast]);
      __syncthreads();
      if (zlast == bv) break;
    }
    for (int i = tid; i < n; i += kThreads)
      x[i] = ((i & 1) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(n - 1));
    __syncthreads();
    apply_power(Acur, AI2, n, p, x, tmp, 0, S.work);
    const double alt = 2.0 * vec_abs_sum(x, n, S.red) / (3.0 * n);
    if (alt > est) est = alt;
  }
  return est;
}

// ---------------------------------------------------------------------------
// alpha_m <= Theta by eqs. (alphaapprox), (normAm9), (alpha2term1),
// (normAm9plus1) of Sec. 6. AI2 == nullptr means s = 0 (powers of B itself).
// ---------------------------------------------------------------------------
struct EstState {
  double t_m, t_m1;
  int m, n_est;
};

__device__ int alpha_test(const double* Acur, const double* AI2, int n, double nB, double nI2, int m,
                          double theta, EstState& st, double* alpha, BlockSmem& S) {
  const double th_m = ipow(theta, m), th_m1 = ipow(theta, m + 1);
  double t1, t2;
  int have_est1 = 0;
  st.m = m;
  st.t_m = -1.0;
  st.t_m1 = -1.0;
  if (AI2 && m == 2) {
    t1 = nI2;
  } else if (AI2 && ipow(nI2, m / 2) <= th_m) {
    t1 = ipow(nI2, m / 2);
  } else {
    t1 = normest_pow(Acur, AI2, n, m, S);
    st.n_est++;
    st.t_m = t1;
    have_est1 = 1;
  }
  if (!(t1 <= th_m)) {
    *alpha = pow(t1, 1.0 / m);
    return 0;
  }
  const double base = have_est1 ? t1 : (AI2 ? ipow(nI2, m / 2) : t1);
  if (base * nB <= th_m1) {
    t2 = base * nB;
  } else {
    t2 = normest_pow(Acur, AI2, n, m + 1, S);
    st.n_est++;
    st.t_m1 = t2;
  }
  const double a1 = pow(t1, 1.0 / m), a2 = pow(t2, 1.0 / (m + 1));
  *alpha = a1 > a2 ? a1 : a2;
  return t2 <= th_m1;
}

// Order search (Step 'StepFinminm' of Algorithm 1, Sec. 6): min_im from the
// loop's estimates (eqs. min_in, min_inp), max_in from the rough bound (eq.
// roughmax_even; every available m_k is even), then an increasing scan that
// takes k+1 at once when alpha_{m_k} is above Theta_k but not above Theta_{k+1}.
__device__ int order_search(const double* Acur, const double* AI2, int n, double nB, double nI2,
                            int k_max, const double* theta, const EstState* loop_est, BlockSmem& S) {
  int cands[3], nc = 0;
  const int all[3] = {1, 2, 5};
  for (int t = 0; t < 3; ++t)
    if (all[t] <= k_max) cands[nc++] = all[t];
  if (nc == 0) return k_max;
  int lo = 0;
  if (loop_est && loop_est->t_m >= 0.0) {
    const int mm = loop_est->m;
    while (lo < nc - 1) {
      const double th = theta[theta_slot(cands[lo])];
      int ok = loop_est->t_m <= ipow(th, mm);
      if (ok && loop_est->t_m1 >= 0.0) ok = loop_est->t_m1 <= ipow(th, mm + 1);
      if (ok) break;
      ++lo;
    }
  }
  int hi = nc - 1;
  for (int t = 0; t < nc; ++t) {
    const int m = m_of_k(cands[t]);
    const double th = theta[theta_slot(cands[t])];
    if (ipow(nI2, m / 2) * nB <= ipow(th, m + 1)) {
      hi = t;
      break;
    }
  }
  if (lo >= hi) return cands[hi];
  for (int t = lo; t < hi; ++t) {
    const int m = m_of_k(cands[t]);
    const double th = theta[theta_slot(cands[t])];
    EstState st{-1.0, -1.0, m, 0};
    double a;
    if (alpha_test(Acur, AI2, n, nB, nI2, m, th, st, &a, S)) return cands[t];
    const double thn = theta[theta_slot(cands[t + 1])];
    const double t1 = (st.t_m >= 0.0) ? st.t_m : (m == 2 ? nI2 : ipow(nI2, m / 2));
    if (t1 <= ipow(thn, m)) {
      double t2 = st.t_m1;
      if (t2 < 0.0) {
        if (t1 * nB <= ipow(thn, m + 1))
          t2 = t1 * nB;
        else
          t2 = normest_pow(Acur, AI2, n, m + 1, S);
      }
      if (t2 <= ipow(thn, m + 1)) return cands[t + 1];
    }
  }
  return cands[hi];
}

// ---------------------------------------------------------------------------
// Scaled Denman-Beavers square root, eq. (ScalDB): X_0 = A (in Acur, in
// place), Y_0 = I, mu_k = |det X_k det Y_k|^{-1/(2n)} from the pivots of the
// two Gauss-Jordan inverses. Stop when the relative 1-norm change of X is
// <= 10 sqrt(n) u, or, once scaling is off and the change has reached 1e-7,
// when it no longer halves; scaling is switched off below 1e-2.
// Returns 0 (converged), 1 (singular) or 2 (no convergence).
// ---------------------------------------------------------------------------
__device__ int db_sqrt(Slot& M, int n, int max_db, int* iters_out, BlockSmem& S) {
  double* X = M.Acur;
  double* Y = M.Y;
  mat_identity(Y, n);
  __syncthreads();
  const double tol = 10.0 * sqrt((double)n) * kUnitRoundoff;
  int scale = 1, status = 2, it;
  double dprev = INFINITY;
  for (it = 1; it <= max_db; ++it) {
    double ldx, ldy;
    if (threadIdx.x == 0) {
      S.work[0] += 1;
      S.work[1] += (it == 1) ? 1 : 2;
    }
    mat_copy(M.W1, X, n);
    __syncthreads();
    if (gj_inverse_block(M.W1, n, &ldx, S)) { status = 1; break; }
    if (it == 1) {
      // Y_0 = I: its inverse is I and log|det Y_0| = 0 exactly.
      mat_identity(M.W2, n);
      ldy = 0.0;
      __syncthreads();
    } else {
      mat_copy(M.W2, Y, n);
      __syncthreads();
      if (gj_inverse_block(M.W2, n, &ldy, S)) { status = 1; break; }
    }
    if (threadIdx.x == 0) {
      const double mu = scale ? exp(-(ldx + ldy) / (2.0 * n)) : 1.0;
      S.bc[2] = mu;
      S.bc[3] = 1.0 / mu;
    }
    __syncthreads();
    const double mu = S.bc[2], imu = S.bc[3];
    double sd = 0.0, sx = 0.0;
    for (int j = threadIdx.x; j < n; j += kThreads) {
      double cd = 0.0, cx = 0.0;
      for (int i = 0; i < n; ++i) {
        const int t = i * n + j;
        const double xo = X[t];
        const double xn = 0.5 * fma(mu, xo, M.W2[t] * imu);
        Y[t] = 0.5 * fma(mu, Y[t], M.W1[t] * imu);
        X[t] = xn;
        cd += fabs(xn - xo);
        cx += fabs(xn);
      }
      sd = nanmax(sd, cd);
      sx = nanmax(sx, cx);
    }
    const double nd = block_max(sd, S.red);
    const double nx = block_max(sx, S.red);
    const double delta = nd / nx;
    if (!(delta == delta)) { status = 2; break; }
    if (delta <= tol) { status = 0; break; }
    if (!scale && dprev <= 1e-7 && delta > 0.5 * dprev) { status = 0; break; }
    if (delta < 1e-2) scale = 0;
    dprev = delta;
  }
  *iters_out = it > max_db ? max_db : it;
  return status;
}

// ---------------------------------------------------------------------------
// Graph evaluation, eq. (five_mult_degopt): out = scale * z(X) with P_2 = X,
// P_3 = X^2 given. For Algorithm 1, scale = -2^s (eq. logipASTM and the final
// squaring step): a power of two, so it changes no rounding.
// ---------------------------------------------------------------------------
__device__ void graph_block(int k, int n, Slot& M, double scale, OutView out, BlockSmem& S) {
  double* P2 = M.Acur;
  double* P3 = M.A2;
  if (k == 1) {  // z = X + X^2/2 (Taylor T_2)
    const int nn = n * n;
    for (int t = threadIdx.x; t < nn; t += kThreads) store_out(out, t, scale * fma(0.5, P3[t], P2[t]));
    __syncthreads();
    return;
  }
  if (k == 2) {  // P_4 = X^2 (X/3 + X^2/4); z = X + X^2/2 + P_4 (Taylor T_4)
    EpiTerms r{{P2, P3}, {1.0 / 3.0, 0.25}, 2};
    lincomb_block(n, r, M.T2);
    EpiTerms e{{P2, P3}, {scale, 0.5 * scale}, 2};
    if (threadIdx.x == 0) S.work[2] += 1;
    gemm_block(n, P3, 0.0, M.T2, 0.0, scale, e, out, S.u.gemm);
    return;
  }
  // k = 5: P_4 .. P_7 from Table table_simple_experiment
  double* P[8] = {nullptr, nullptr, P2, P3, M.Y, M.W1, M.W2, nullptr};
  int t = 0;
  for (int j = 2; j <= 5; ++j) {
    EpiTerms hl, gl;
    hl.count = gl.count = j;
    for (int i = 2; i <= j + 1; ++i, ++t) {
      hl.M[i - 2] = P[i];
      hl.c[i - 2] = c_h5[t];
      gl.M[i - 2] = P[i];
      gl.c[i - 2] = c_g5[t];
    }
    lincomb_block(n, hl, M.T1);
    lincomb_block(n, gl, M.T2);
    if (threadIdx.x == 0) S.work[2] += 1;
    if (j < 5) {
      EpiTerms none;
      none.count = 0;
      gemm_block(n, M.T1, 0.0, M.T2, 0.0, 1.0, none, OutView{P[j + 2], 0}, S.u.gemm);
    } else {
      EpiTerms e;
      e.count = 5;
      for (int i = 2; i <= 6; ++i) {
        e.M[i - 2] = P[i];
        e.c[i - 2] = scale * c_y5[i - 1];
      }
      gemm_block(n, M.T1, 0.0, M.T2, 0.0, scale * c_y5[6], e, out, S.u.gemm);
    }
  }
}

// ---------------------------------------------------------------------------
// One matrix per block, per mode.
// ---------------------------------------------------------------------------
__device__ void matrix_geometry(const SmallParams& p, int b, int* n, int64_t* off) {
  if (p.n_uniform > 0) {
    *n = p.n_uniform;
    *off = (int64_t)b * p.n_uniform * p.n_uniform;
  } else {
    *n = p.n_dev[b];
    *off = p.off_dev[b];
  }
}

__device__ void ai2_from(Slot& M, int n) {
  // A_I2 = A_2 - 2A + I (eq. AI2), written over A_2.
  const int nn = n * n;
  for (int t = threadIdx.x; t < nn; t += kThreads) {
    double v = M.A2[t] - 2.0 * M.Acur[t];
    if (t / n == t % n) v += 1.0;
    M.A2[t] = v;
  }
  __syncthreads();
}

__device__ void run_execute(const SmallParams& p, int b, Slot& M, BlockSmem& S) {
  int n;
  int64_t off;
  matrix_geometry(p, b, &n, &off);
  const int km = p.k_max;
  if (n < 1 || n > kMaxN || n > p.n_max) {
    if (threadIdx.x == 0) {
      p.info[b] = -1;
      if (p.s_out) p.s_out[b] = 0;
      if (p.k_out) p.k_out[b] = km;
    }
    return;
  }
  if (threadIdx.x == 0) S.work[0] = S.work[1] = S.work[2] = S.work[3] = 0;
  const int finite = load_matrix(p.A, p.dtype, off, n, M.Acur, S.red);
  if (!finite) {
    fill_nan(p.L, p.dtype, off, n);
    if (threadIdx.x == 0) {
      if (p.stats)
        for (int t = 0; t < 4; ++t) p.stats[4 * b + t] = 0;
      p.info[b] = 4;
      if (p.s_out) p.s_out[b] = 0;
      if (p.k_out) p.k_out[b] = km;
    }
    return;
  }
  const int m = m_of_k(km);
  const double th = p.theta[theta_slot(km)];
  double nB = mat_norm1(M.Acur, n, 1.0, S.red), nI2 = 0.0;
  int s = 0, have_ai2 = 0, info = 0, finish = nB <= th;
  double alpha = nB;
  EstState last{-1.0, -1.0, m, 0};
  while (!finish && s < p.max_sqrt) {
    EstState st{-1.0, -1.0, m, 0};
    finish = alpha_test(M.Acur, have_ai2 ? M.A2 : nullptr, n, nB, nI2, m, th, st, &alpha, S);
    last = st;
    if (finish) break;
    if (p.ctx && s < p.ctx_levels) {
      double* ck = p.ctx + ((int64_t)b * p.ctx_levels + s) * (int64_t)p.n_max * p.n_max;
      mat_copy(ck, M.Acur, n);
    }
    mat_copy(M.A2, M.Acur, n);
    __syncthreads();
    int it;
    const int r = db_sqrt(M, n, p.max_db, &it, S);
    if (r == 1) { info = 1; break; }
    if (r == 2 && info == 0) info = 2;
    ai2_from(M, n);
    nB = mat_norm1(M.Acur, n, 1.0, S.red);
    nI2 = mat_norm1(M.A2, n, 0.0, S.red);
    have_ai2 = 1;
    ++s;
  }
  int k = km;
  if (info == 1) {
    fill_nan(p.L, p.dtype, off, n);
  } else {
    if (!finish && info == 0) info = 3;
    if (!have_ai2) {
      EpiTerms none;
      none.count = 0;
      if (threadIdx.x == 0) S.work[2] += 1;
      gemm_block(n, M.Acur, 1.0, M.Acur, 1.0, 1.0, none, OutView{M.A2, 0}, S.u.gemm);
      nI2 = mat_norm1(M.A2, n, 0.0, S.red);
    }
    if (finish)
      k = order_search(M.Acur, M.A2, n, nB, nI2, km, p.theta, last.t_m >= 0.0 ? &last : nullptr, S);
    // P_2 = X = -(A - I)
    const int nn = n * n;
    for (int t = threadIdx.x; t < nn; t += kThreads) {
      double v = M.Acur[t];
      if (t / n == t % n) v -= 1.0;
      M.Acur[t] = -v;
    }
    __syncthreads();
    graph_block(k, n, M, -ldexp(1.0, s), out_view(p.L, p.dtype, off), S);
  }
  if (threadIdx.x == 0) {
    p.info[b] = info;
    if (p.s_out) p.s_out[b] = s;
    if (p.k_out) p.k_out[b] = k;
    if (p.alpha) p.alpha[b] = alpha;
    if (p.stats)
      for (int t = 0; t < 4; ++t) p.stats[4 * b + t] = S.work[t];
  }
}

__device__ void run_plan(const SmallParams& p, int b, Slot& M, BlockSmem& S) {
  int n;
  int64_t off;
  matrix_geometry(p, b, &n, &off);
  const int km = p.k_max;
  if (n < 1 || n > kMaxN || n > p.n_max) {
    if (threadIdx.x == 0) p.info[b] = -1;
    return;
  }
  const int finite = load_matrix(p.A, p.dtype, off, n, M.Acur, S.red);
  int fin2 = 1;
  if (p.AI2_in) fin2 = load_matrix(p.AI2_in, p.dtype, off, n, M.A2, S.red);
  if (!finite || !fin2) {
    if (threadIdx.x == 0) {
      p.info[b] = 4;
      p.finish[b] = 0;
      p.k_out[b] = km;
      p.alpha[b] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  const int m = m_of_k(km);
  const double th = p.theta[theta_slot(km)];
  const double nB = mat_norm1(M.Acur, n, 1.0, S.red);
  EstState st{-1.0, -1.0, m, 0};
  int fin;
  double a;
  double nI2 = p.AI2_in ? mat_norm1(M.A2, n, 0.0, S.red) : 0.0;
  if (!p.AI2_in && nB <= th) {
    fin = 1;
    a = nB;
  } else {
    fin = alpha_test(M.Acur, p.AI2_in ? M.A2 : nullptr, n, nB, nI2, m, th, st, &a, S);
  }
  if (!p.AI2_in) {
    EpiTerms none;
    none.count = 0;
    gemm_block(n, M.Acur, 1.0, M.Acur, 1.0, 1.0, none, OutView{M.A2, 0}, S.u.gemm);
    nI2 = mat_norm1(M.A2, n, 0.0, S.red);
  }
  const int k = fin ? order_search(M.Acur, M.A2, n, nB, nI2, km, p.theta, &st, S) : km;
  if (threadIdx.x == 0) {
    p.info[b] = 0;
    p.finish[b] = fin;
    p.k_out[b] = k;
    p.alpha[b] = a;
  }
}

__device__ void run_sqrt(const SmallParams& p, int b, Slot& M, BlockSmem& S) {
  int n;
  int64_t off;
  matrix_geometry(p, b, &n, &off);
  if (p.active && p.active[b] == 0) {
    if (threadIdx.x == 0) {
      p.info[b] = 0;
      if (p.iters) p.iters[b] = 0;
    }
    return;
  }
  if (n < 1 || n > kMaxN || n > p.n_max) {
    if (threadIdx.x == 0) p.info[b] = -1;
    return;
  }
  const int finite = load_matrix(p.A_inout, p.dtype, off, n, M.Acur, S.red);
  if (!finite) {
    if (threadIdx.x == 0) {
      p.info[b] = 4;
      if (p.iters) p.iters[b] = 0;
    }
    return;
  }
  mat_copy(M.A2, M.Acur, n);
  __syncthreads();
  if (p.A2_out) store_matrix(p.A2_out, p.dtype, off, n, M.A2);
  int it;
  const int r = db_sqrt(M, n, p.max_db, &it, S);
  store_matrix(p.A_inout, p.dtype, off, n, M.Acur);
  if (p.AI2_out) {
    ai2_from(M, n);
    store_matrix(p.AI2_out, p.dtype, off, n, M.A2);
  }
  if (threadIdx.x == 0) {
    p.info[b] = r;
    if (p.iters) p.iters[b] = it;
  }
}

__device__ void run_graph(const SmallParams& p, int b, Slot& M, BlockSmem& S) {
  int n;
  int64_t off;
  matrix_geometry(p, b, &n, &off);
  const int k = p.k_in[b];
  if (n < 1 || n > kMaxN || n > p.n_max || !(k == 1 || k == 2 || k == 5)) {
    if (threadIdx.x == 0 && p.info) p.info[b] = -1;
    return;
  }
  load_matrix(p.X, p.dtype, off, n, M.Acur, S.red);
  if (p.P3) {
    load_matrix(p.P3, p.dtype, off, n, M.A2, S.red);
  } else {
    EpiTerms none;
    none.count = 0;
    gemm_block(n, M.Acur, 0.0, M.Acur, 0.0, 1.0, none, OutView{M.A2, 0}, S.u.gemm);
  }
  graph_block(k, n, M, 1.0, out_view(p.L, p.dtype, off), S);
  if (threadIdx.x == 0 && p.info) p.info[b] = 0;
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
  const double th = p.theta[theta_slot(p.k_max)];
  for (int b = blockIdx.x; b < p.count; b += gridDim.x) {
    int n;
    int64_t off;
    matrix_geometry(p, b, &n, &off);
    double best = 0.0;
    if (n >= 1 && n <= p.n_max) {
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
      const double n3 = (n >= 1 ? (double)n * n * n : 1.0);
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
__global__ void __launch_bounds__(kThreads, 2) k_logm_small(SmallParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSmem& S = *reinterpret_cast<BlockSmem*>(smem_raw);
  const int64_t nn_max = (int64_t)p.n_max * p.n_max;
  double* base = p.slots + (int64_t)blockIdx.x * kSlotMats * nn_max;
  Slot M{base, base + nn_max, base + 2 * nn_max, base + 3 * nn_max,
         base + 4 * nn_max, base + 5 * nn_max, base + 6 * nn_max};
  for (;;) {
    if (threadIdx.x == 0) S.ibc[0] = atomicAdd(p.queue, 1);
    __syncthreads();
    const int q = S.ibc[0];
    __syncthreads();
    if (q >= p.count) break;
    const int b = p.order ? p.order[q] : q;
    if (threadIdx.x == 0) S.work[0] = S.work[1] = S.work[2] = S.work[3] = 0;
    if (MODE == kModeExecute) run_execute(p, b, M, S);
    if (MODE == kModePlan) run_plan(p, b, M, S);
    if (MODE == kModeSqrt) run_sqrt(p, b, M, S);
    if (MODE == kModeGraph) run_graph(p, b, M, S);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int g_sm_count = 0;

static int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 1;
  }
  return g_sm_count;
}

int small_kernel_slots(int count) {
  const int per_sm = 2;  // blocks resident per SM (shared memory and registers)
  const int cap = sm_count() * per_sm;
  return count < cap ? (count > 0 ? count : 1) : cap;
}

size_t small_order_bytes(int count) {
  const size_t raw = sizeof(int32_t) * ((size_t)count + 2 * kOrderBuckets + (size_t)count);
  return (raw + 255) / 256 * 256;
}

size_t small_workspace_bytes(int count, int n_max) {
  const size_t slots = (size_t)small_kernel_slots(count);
  return 256 + small_order_bytes(count) + slots * kSlotMats * (size_t)n_max * n_max * sizeof(double);
}

template <int MODE>
static cudaError_t launch_mode(const SmallParams& p, cudaStream_t st) {
  static bool attr_set = false;
  const size_t smem = sizeof(BlockSmem);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_logm_small<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaError_t e = cudaMemsetAsync(p.queue, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  if (MODE == kModeExecute && p.order && p.order_aux && p.count > 1) {
    e = cudaMemsetAsync(p.order_aux, 0, sizeof(int32_t) * 2 * kOrderBuckets, st);
    if (e != cudaSuccess) return e;
    const int kb = p.count < 4 * sm_count() ? p.count : 4 * sm_count();
    k_order_keys<<<kb, kThreads, 0, st>>>(p);
    k_order_scan<<<1, 32, 0, st>>>(p);
    k_order_scatter<<<(p.count + kThreads - 1) / kThreads, kThreads, 0, st>>>(p);
  }
  SmallParams q = p;
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
  }
  return cudaErrorInvalidValue;
}

}  // namespace lg
