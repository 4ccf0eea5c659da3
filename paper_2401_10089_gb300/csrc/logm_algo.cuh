// logm_algo.cuh -- Algorithm 1 of arXiv 2401.10089 (Sec. 6), written once
// against an "ops" layer so that the same plan logic, square-root iteration
// and graph evaluation run on one thread block per matrix (BlockOps, n <= 256)
// and on the whole GPU per matrix (GridOps, large n).
//
// An Ops type provides: tid()/nthreads() for strided loops over the
// participating threads, sync(), block-or-grid reductions sum/max/all/argmax
// whose results are bitwise identical in every participating thread,
// bcast0() (a scalar computed by thread 0 of each block), n-vectors vec(i),
// norm1, matvec, gemm, lincomb and an in-place inverse, plus leader() and
// tally() for the per-matrix outputs.
//
// Every branch below depends only on such uniform values, so all threads
// (and, in the grid version, all blocks) take the same path.
#pragma once

#include <cstdint>

#include "cta_linalg.cuh"
#include "logm_internal.h"

namespace LG_NS {

// Table table_simple_experiment (Sec. 3): the k = 5 scheme fitted to
// -log(1 - x). h_{j,i}, g_{j,i} for j = 2..5, i = 2..j+1 in that order.
static __constant__ double c_h5[14] = {
    7.363757032799957e-02, -1.050281301619960e+00, 8.897468955192446e-02,
    -1.599651928992725e-01, 9.577281350989334e-01, 5.394999133948797e-01,
    6.700731102561937e-02, -5.158769100223212e-02, 1.094308587350110e+00,
    1.027072285939197e-01, -8.964023050065877e-03, -2.100705663612491e-01,
    1.949655359168707e-01, 1.117368056772713e+00};
static __constant__ double c_g5[14] = {
    -9.666134174379001e-01, -4.395519034717933e-01, 1.048664069004776e-01,
    1.585606124033259e-01, 1.668066506920988e-01, -8.025600931705978e-02,
    -1.159854366397558e-01, 1.066554944706011e-01, 1.127094008297975e+00,
    2.702180425508705e-01, 4.137541209720699e-02, 4.857347452405025e-01,
    -6.000256005636980e-01, 1.063393233943084e+00};
// y_1 .. y_7 (y_1 = 0: no identity term)
static __constant__ double c_y5[7] = {0.0, 1.0, 5.065546620208965e-01, 3.832512052972577e-01,
                               1.088307723749078e+00, 2.787461897212877e-01,
                               8.157421998489228e-01};

// k = 4, the 14+ scheme of Sec. 3 (m = 14+, degree 16; the paper gives no
// coefficients): P_4 = P_3 (c3 X + c4 P_3), P_5 = (d1 X + d2 P_3 + P_4)
// (e2 P_3 + P_4), P_6 = (f1 X + f2 P_3 + f4 P_4 + P_5)(g1 X + g4 P_4 + P_5),
// z = X + y3 P_3 + y4 P_4 + y5 P_5 + P_6. The 13 values solve "coefficient of
// x^i = 1/i" for i = 2..14 (T_14 of eq. Taylor_log matched; x^15, x^16 are
// the "+"), the real root with the smallest coefficients, correctly rounded
// from a 50-digit solution; Theta_14 recomputed from them is 9.32e-2 (Table
// Table_theta: 9.31e-2). Order: c3 c4 d1 d2 e2 f1 f2 f4 g1 g4 y3 y4 y5.
static __constant__ double c_k4[13] = {
    0.3602750956560524,  0.3018442985303789,   0.3412287952056341,  -0.18047064940974122,
    0.18907274365286242, -0.014079460349863975, 0.24400741065645315, -0.8525627910338015,
    0.1463535711919622,  0.9787518426666669,   0.5020605793026582,  0.6095606808527384,
    1.2091753609836204};

// k = 6 (m_6 = 20+, degree 64, Theta_6 = 0.372 of Table Table_theta), taken
// by the one-block-per-matrix kernels only (LG_WITH_K6 = 1). The paper prints
// no coefficients for k >= 6; these were fitted to -log(1 - x) in the same
// degree-optimal form (P_3 = X^2, y_1 = 0, y_2 = 1), with the Taylor terms
// matched to order 34 and the backward-error Theta of eqs. (Eb), (theta_Eb)
// above 0.372. h_{j,i}, g_{j,i} for j = 2..6, i = 2..j+1 in that order;
// y_3 .. y_8.
#ifndef LG_WITH_K6
#define LG_WITH_K6 0
#endif
#if LG_WITH_K6
static __constant__ double c_h6[20] = {
    -0.03542133528022389, 0.5305162167939017, 1.1735695507060024, 0.42664399607790565,
    -1.4401144598828934, -0.37722719586021003, 1.1748267828138759, -0.4355749562164976,
    -0.55350435103941, -0.13552704716524286, 0.483097031151113, -2.879391574437424,
    -0.779847925333845, -0.8268140965713336, 4.549413425481621, -3.6536822467517673,
    -5.744611071943747, 3.2747363248058474, -3.4999222429973935, 5.3137561222344525};
static __constant__ double c_g6[20] = {
    -0.25821891505961464, -0.5021334801772399, 1.1247378095155132, -0.7530860083722153,
    2.656179396111579, -0.5198936929205077, -0.669272512275526, -1.2980185589839237,
    0.5165656321507225, 0.1625662254422074, -0.2675459778240617, -0.03466835614054706,
    0.328082088789197, -0.34992616877127714, -1.3970630865902485, 2.542415746918083,
    -0.048059210298082834, 0.9420478294952318, -2.416723959179748, 1.3390816588113656};
static __constant__ double c_y6[6] = {0.8200410102947662,   -0.4825318072757668, -0.12989653721591463,
                                      -0.40476811140333024, 0.12143584229947445, 0.00977242585180227};
constexpr double kTheta6 = kThetaPaper[5];
#endif

constexpr double kUnitRoundoff = 0x1p-53;

struct Slot {
  double *Acur, *A2, *Y, *W1, *W2, *T1, *T2;
};

static __device__ __forceinline__ int m_of_k(int k) { return k == 1 ? 2 : (k == 2 ? 4 : (k == 3 ? 8 : 14)); }
static __device__ __forceinline__ int theta_slot(int k) { return k - 1; }

// m_k (LG_M_OF) and Theta_{m_k} (LG_THETA) of order k, and the largest order
// (LG_MAX_ORDER). Theta_1..Theta_5 come from the caller's options (theta[0..4]);
// Theta_6 is the table's. Without k = 6 these are the plain table lookups.
#if LG_WITH_K6
static __device__ __forceinline__ int m_of_order(int k) { return k == 6 ? 20 : m_of_k(k); }
static __device__ __forceinline__ double theta_of(const double* theta, int k) {
  return k == 6 ? kTheta6 : theta[theta_slot(k)];
}
#define LG_M_OF(k) m_of_order(k)
#define LG_THETA(th, k) theta_of(th, k)
#define LG_MAX_ORDER 6
#else
#define LG_M_OF(k) m_of_k(k)
#define LG_THETA(th, k) th[theta_slot(k)]
#define LG_MAX_ORDER 5
#endif

// k = 3 (Sec. 2, eq. eqP8pol): T_8 of eq. (Taylor_log) with three products,
//   y02 = X^2 (c4 X^2 + c3 X),
//   z   = (y02 + d2 X^2 + d1 X)(y02 + e2 X^2) + e0 y02 + X^2/2 + X.
// Equating the coefficients of x^8 .. x^3 with 1/8 .. 1/3 fixes, in turn,
// c4 = 1/sqrt(8), c3 = 1/(14 c4), d2 + e2 = S, d1, and leaves a quadratic in
// e2; the root with the smaller coefficients is taken (it also rounds better:
// its monomials match 1/i within about 1.3 u). c = c3, c4, d1, d2, e2, e0.
static __device__ void k3_coeffs(double* c) {
  const double c4 = 1.0 / sqrt(8.0);
  const double c3 = 1.0 / (14.0 * c4);
  const double sum = (1.0 / 6.0 - c3 * c3) / c4;  // d2 + e2
  const double d1 = (1.0 / 5.0 - c3 * sum) / c4;
  const double beta = sum - c4 * d1 / c3;
  const double gamma = c3 * d1 + c4 / (3.0 * c3) - 0.25;
  const double e2 = 0.5 * (beta + sqrt(beta * beta + 4.0 * gamma));
  c[0] = c3;
  c[1] = c4;
  c[2] = d1;
  c[3] = sum - e2;
  c[4] = e2;
  c[5] = (1.0 / 3.0 - d1 * e2) / c3;
}

// x^m by repeated multiplication, so that "x^{1/m} <= Theta" is decided as
// "x <= Theta^m" exactly the same way in every implementation.
static __device__ __forceinline__ double ipow(double x, int m) {
  double r = 1.0;
  for (int i = 0; i < m; ++i) r *= x;
  return r;
}

static __device__ __forceinline__ double load_elem(const void* base, int dtype, int64_t idx) {
  return dtype == 0 ? static_cast<const double*>(base)[idx]
                    : static_cast<double>(static_cast<const float*>(base)[idx]);
}

static __device__ __forceinline__ OutView out_view(void* base, int dtype, int64_t off) {
  return OutView{dtype == 0 ? static_cast<void*>(static_cast<double*>(base) + off)
                            : static_cast<void*>(static_cast<float*>(base) + off),
                 dtype};
}

static __device__ __forceinline__ void matrix_geometry(const SmallParams& p, int b, int* n, int64_t* off) {
  if (p.n_uniform > 0) {
    *n = p.n_uniform;
    *off = (int64_t)b * p.n_uniform * p.n_uniform;
  } else {
    *n = p.n_dev[b];
    *off = p.off_dev[b];
  }
}

// ---------------------------------------------------------------------------
// Elementwise steps
// ---------------------------------------------------------------------------
template <class Ops>
static __device__ int load_matrix(Ops& ops, const void* src, int dtype, int64_t off, int n, double* dst) {
  int ok = 1;
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) {
    const double v = load_elem(src, dtype, off + t);
    ok &= isfinite(v) ? 1 : 0;
    dst[t] = v;
  }
  return ops.all(ok);  // also orders the stores before later reads
}

template <class Ops>
static __device__ void store_matrix(Ops& ops, void* dst, int dtype, int64_t off, int n, const double* src) {
  const OutView o = out_view(dst, dtype, off);
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) store_out(o, t, src[t]);
  ops.sync();
}

template <class Ops>
static __device__ void fill_nan(Ops& ops, void* dst, int dtype, int64_t off, int n) {
  const OutView o = out_view(dst, dtype, off);
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads())
    store_out(o, t, __longlong_as_double(0x7ff8000000000000ll));
  ops.sync();
}

template <class Ops>
static __device__ void copy_matrix(Ops& ops, double* dst, const double* src, int n) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) dst[t] = src[t];
  ops.sync();
}

template <class Ops>
static __device__ void identity_matrix(Ops& ops, double* dst, int n) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) dst[t] = (t / n == t % n) ? 1.0 : 0.0;
  ops.sync();
}

// A_I2 = A_2 - 2A + I (eq. AI2), written over A_2.
template <class Ops>
static __device__ void ai2_from(Ops& ops, Slot& M, int n) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) {
    double v = M.A2[t] - 2.0 * M.Acur[t];
    if (t / n == t % n) v += 1.0;
    M.A2[t] = v;
  }
  ops.sync();
}

// X = -(A - I), in place.
template <class Ops>
static __device__ void to_x(Ops& ops, double* A, int n) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) {
    double v = A[t];
    if (t / n == t % n) v -= 1.0;
    A[t] = -v;
  }
  ops.sync();
}

// ---------------------------------------------------------------------------
// 1-norm estimate of ||B^p||_1, B = Acur - I (Higham 1988, the estimator the
// paper cites in Sec. 6). With A_I2 = B^2 (eq. AI2) the power is applied as
// B^{p mod 2} A_I2^{p div 2} (Sec. 6, item 2). One vector, at most 5 sweeps,
// ties to the smallest index, sign(0) = +1, then the alternating-sign test.
// ---------------------------------------------------------------------------
template <class Ops>
static __device__ void apply_power(Ops& ops, const double* Acur, const double* AI2, int n, int p, double* v,
                            double* tmp, int trans) {
  const int q = AI2 ? (p & 1) : p;
  const int r = AI2 ? (p >> 1) : 0;
  ops.tally(3, q + r);
  double* cur = v;
  double* oth = tmp;
  if (!trans) {
    for (int t = 0; t < r; ++t) {
      ops.matvec(AI2, n, 0.0, cur, oth, 0);
      double* s = cur; cur = oth; oth = s;
    }
    for (int t = 0; t < q; ++t) {
      ops.matvec(Acur, n, 1.0, cur, oth, 0);
      double* s = cur; cur = oth; oth = s;
    }
  } else {
    for (int t = 0; t < q; ++t) {
      ops.matvec(Acur, n, 1.0, cur, oth, 1);
      double* s = cur; cur = oth; oth = s;
    }
    for (int t = 0; t < r; ++t) {
      ops.matvec(AI2, n, 0.0, cur, oth, 1);
      double* s = cur; cur = oth; oth = s;
    }
  }
  if (cur != v) {
    for (int i = ops.tid(); i < n; i += ops.nthreads()) v[i] = cur[i];
    ops.sync();
  }
}

template <class Ops>
static __device__ void argmax_abs(Ops& ops, const double* x, int n, double* bv, int* j) {
  double cv = -1.0;
  int ci = n;
  for (int i = ops.tid(); i < n; i += ops.nthreads()) {
    const double a = fabs(x[i]);
    if (a > cv) { cv = a; ci = i; }
  }
  ops.argmax(cv, ci, bv, j);
}

template <class Ops>
static __device__ double normest_pow(Ops& ops, const double* Acur, const double* AI2, int n, int p) {
  double* x = ops.vec(0);
  double* tmp = ops.vec(1);
  double* xi = ops.vec(2);
  for (int i = ops.tid(); i < n; i += ops.nthreads()) x[i] = 1.0 / n;
  ops.sync();
  apply_power(ops, Acur, AI2, n, p, x, tmp, 0);
  double s0 = 0.0;
  for (int i = ops.tid(); i < n; i += ops.nthreads()) s0 += fabs(x[i]);
  double est = ops.sum(s0);
  if (n > 1) {
    for (int i = ops.tid(); i < n; i += ops.nthreads()) {
      xi[i] = (x[i] >= 0.0) ? 1.0 : -1.0;
      x[i] = xi[i];
    }
    ops.sync();
    apply_power(ops, Acur, AI2, n, p, x, tmp, 1);
    double bv;
    int j;
    argmax_abs(ops, x, n, &bv, &j);
    for (int sweep = 2; sweep <= 5; ++sweep) {
      ops.sync();  // everyone has read x before it is overwritten
      for (int i = ops.tid(); i < n; i += ops.nthreads()) x[i] = (i == j) ? 1.0 : 0.0;
      ops.sync();
      apply_power(ops, Acur, AI2, n, p, x, tmp, 0);
      double sn = 0.0;
      int same = 1;
      for (int i = ops.tid(); i < n; i += ops.nthreads()) {
        sn += fabs(x[i]);
        same &= (((x[i] >= 0.0) ? 1.0 : -1.0) == xi[i]);
      }
      const double est_new = ops.sum(sn);
      same = ops.all(same);
      if (same || est_new <= est) {
        if (est_new > est) est = est_new;
        break;
      }
      est = est_new;
      for (int i = ops.tid(); i < n; i += ops.nthreads()) {
        xi[i] = (x[i] >= 0.0) ? 1.0 : -1.0;
        x[i] = xi[i];
      }
      ops.sync();
      apply_power(ops, Acur, AI2, n, p, x, tmp, 1);
      const int jlast = j;
      argmax_abs(ops, x, n, &bv, &j);
      const double zlast = fabs(x[jlast]);
      if (zlast == bv) break;
    }
    ops.sync();
    for (int i = ops.tid(); i < n; i += ops.nthreads())
      x[i] = ((i & 1) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(n - 1));
    ops.sync();
    apply_power(ops, Acur, AI2, n, p, x, tmp, 0);
    double sa = 0.0;
    for (int i = ops.tid(); i < n; i += ops.nthreads()) sa += fabs(x[i]);
    const double alt = 2.0 * ops.sum(sa) / (3.0 * n);
    if (alt > est) est = alt;
  }
  ops.sync();
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

template <class Ops>
static __device__ int alpha_test(Ops& ops, const double* Acur, const double* AI2, int n, double nB, double nI2,
                          int m, double theta, EstState& st, double* alpha) {
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
    t1 = normest_pow(ops, Acur, AI2, n, m);
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
    t2 = normest_pow(ops, Acur, AI2, n, m + 1);
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
template <class Ops>
static __device__ int order_search(Ops& ops, const double* Acur, const double* AI2, int n, double nB, double nI2,
                            int k_max, const double* theta, const EstState* loop_est) {
  int cands[LG_MAX_ORDER], nc = 0;
  for (int kk = 1; kk <= LG_MAX_ORDER; ++kk)
    if (kk <= k_max) cands[nc++] = kk;
  if (nc == 0) return k_max;
  int lo = 0;
  if (loop_est && loop_est->t_m >= 0.0) {
    const int mm = loop_est->m;
    while (lo < nc - 1) {
      const double th = LG_THETA(theta, cands[lo]);
      int ok = loop_est->t_m <= ipow(th, mm);
      if (ok && loop_est->t_m1 >= 0.0) ok = loop_est->t_m1 <= ipow(th, mm + 1);
      if (ok) break;
      ++lo;
    }
  }
  int hi = nc - 1;
  for (int t = 0; t < nc; ++t) {
    const int m = LG_M_OF(cands[t]);
    const double th = LG_THETA(theta, cands[t]);
    if (ipow(nI2, m / 2) * nB <= ipow(th, m + 1)) {
      hi = t;
      break;
    }
  }
  if (lo >= hi) return cands[hi];
  for (int t = lo; t < hi; ++t) {
    const int m = LG_M_OF(cands[t]);
    const double th = LG_THETA(theta, cands[t]);
    EstState st{-1.0, -1.0, m, 0};
    double a;
    if (alpha_test(ops, Acur, AI2, n, nB, nI2, m, th, st, &a)) return cands[t];
    const double thn = LG_THETA(theta, cands[t + 1]);
    const double t1 = (st.t_m >= 0.0) ? st.t_m : (m == 2 ? nI2 : ipow(nI2, m / 2));
    if (t1 <= ipow(thn, m)) {
      double t2 = st.t_m1;
      if (t2 < 0.0) {
        if (t1 * nB <= ipow(thn, m + 1))
          t2 = t1 * nB;
        else
          t2 = normest_pow(ops, Acur, AI2, n, m + 1);
      }
      if (t2 <= ipow(thn, m + 1)) return cands[t + 1];
    }
  }
  return cands[hi];
}

// ---------------------------------------------------------------------------
// Scaled Denman-Beavers square root, eq. (ScalDB): X_0 = A (in Acur, in
// place), Y_0 = I, mu_k = |det X_k det Y_k|^{-1/(2n)} from the pivots of the
// two inverses. With delta the relative 1-norm change of X and tol =
// 10 sqrt(n) u: stop when delta <= tol; or, once scaling is off (mu = 1, a
// Newton step, quadratically convergent), when delta^2 ||X_k^{-1}|| ||X_{k+1}||
// <= tol, the relative error that step leaves, so that no step is spent only
// confirming convergence; or, once scaling is off and delta has reached
// 1e-7, when it no longer halves. Scaling is switched off below 1e-2.
// Returns 0 (converged), 1 (singular) or 2 (no convergence).
// ---------------------------------------------------------------------------
// Optional record of one square root for the adjoint: X_i^{-1}, Y_i^{-1} and
// mu_i of every iteration i (the inverses are written straight into the tape).
struct DbTape {
  double* inv;     // [cap][2][stride]
  double* mu;      // [cap]
  int64_t stride;  // n_max^2
  int cap;
};

template <class Ops>
static __device__ int db_sqrt(Ops& ops, Slot& M, int n, int max_db, int* iters_out, const DbTape* tape = nullptr,
                              int reuse = 0, double* ld_io = nullptr) {
  double* X = M.Acur;
  double* Y = M.Y;
  // reuse (a root of the previous level's root, no tape): M.Y still holds the
  // previous level's converged Y, which is A^{-1} of this level's A; it stands
  // in for the first step's inversion, and *ld_io holds log|det A|
  if (reuse) copy_matrix(ops, M.W1, Y, n);
  identity_matrix(ops, Y, n);
  const double tol = 10.0 * sqrt((double)n) * kUnitRoundoff;
  int scale = 1, status = 2, it;
  double dprev = INFINITY;
  for (it = 1; it <= max_db; ++it) {
    double ldx, ldy;
    ops.tally(0, 1);
    ops.tally(1, (it == 1) ? (reuse ? 0 : 1) : 2);
    const bool taped = tape && it - 1 < tape->cap;
    double* Xi = taped ? tape->inv + (int64_t)(2 * (it - 1)) * tape->stride : M.W1;
    double* Yi = taped ? tape->inv + (int64_t)(2 * (it - 1) + 1) * tape->stride : M.W2;
    if (it == 1) {
      if (reuse) {
        ldx = *ld_io;  // Xi (= M.W1) was filled above
      } else if (ops.inverse(X, Xi, n, &ldx)) {
        status = 1;
        break;
      }
      if (ld_io) *ld_io = 0.5 * ldx;  // log|det| of the root, for the next level
      // Y_0 = I: its inverse is I and log|det Y_0| = 0 exactly.
      identity_matrix(ops, Yi, n);
      ldy = 0.0;
    } else {
      if (ops.inverse_pair(X, Xi, Y, Yi, n, &ldx, &ldy)) { status = 1; break; }
    }
    const double mu = ops.bcast0(scale ? exp(-(ldx + ldy) / (2.0 * n)) : 1.0);
    const double imu = ops.bcast0(1.0 / mu);
    if (taped && ops.leader()) tape->mu[it - 1] = mu;
    double nd, nx;
    ops.db_update(X, Y, Xi, Yi, mu, imu, n, &nd, &nx);
    const double delta = nd / nx;
    if (!(delta == delta)) { status = 2; break; }
    if (delta <= tol) { status = 0; break; }
    if (!scale && delta * delta * ops.norm1(Xi, n, 0.0) * nx <= tol) { status = 0; break; }
    if (!scale && dprev <= 1e-7 && delta > 0.5 * dprev) { status = 0; break; }
    if (delta < 1e-2) scale = 0;
    dprev = delta;
  }
  *iters_out = it > max_db ? max_db : it;
  return status;
}

// ---------------------------------------------------------------------------
// Product form of the scaled Denman-Beavers iteration (the variant cited in
// Sec. 2): with M_k = X_k Y_k the two inversions of eq. (ScalDB) become one,
//   M_{k+1} = I/2 + (mu_k^2 M_k + mu_k^{-2} M_k^{-1}) / 4,
//   X_{k+1} = (mu_k X_k + mu_k^{-1} X_k M_k^{-1}) / 2,
// M_0 = X_0 = A, mu_k = |det M_k|^{-1/(2n)}: one inversion and one product
// per step (none in the first: X_0 M_0^{-1} = I). Same stop rule, with the
// error left by a step bounded through M_k instead of X_k^{-1}. X lives in
// Acur, M in Y, M^{-1} in W1, X M^{-1} in W2 (A2 is left alone).
// ---------------------------------------------------------------------------
template <class Ops>
static __device__ int db_sqrt_product(Ops& ops, Slot& M, int n, int max_db, int* iters_out) {
  double* X = M.Acur;
  double* Mk = M.Y;
  double* Mi = M.W1;
  double* XMi = M.W2;
  copy_matrix(ops, Mk, X, n);
  const double tol = 10.0 * sqrt((double)n) * kUnitRoundoff;
  int scale = 1, status = 2, it;
  double dprev = INFINITY;
  for (it = 1; it <= max_db; ++it) {
    double ldm;
    ops.tally(0, 1);
    ops.tally(1, 1);
    if (ops.inverse(Mk, Mi, n, &ldm)) { status = 1; break; }
    const double mu = ops.bcast0(scale ? exp(-ldm / (2.0 * n)) : 1.0);
    const double imu = ops.bcast0(1.0 / mu);
    const double mu2 = ops.bcast0(mu * mu);
    const double imu2 = ops.bcast0(imu * imu);
    // With mu = 1, M_{k+1} - I = M_k^{-1} (M_k - I)^2 / 4 and X_{k+1} ~ X_* M_{k+1}^{1/2}:
    // the step leaves a relative error <= ||M_k^{-1}|| ||M_k||^2 ||I - M_k^{-1}||^2 / 8.
    double pred = INFINITY;
    if (!scale) {
      const double nm = ops.norm1(Mk, n, 0.0), nmi = ops.norm1(Mi, n, 0.0), d = ops.norm1(Mi, n, 1.0);
      pred = 0.125 * nmi * nm * nm * d * d;
    }
    if (it > 1) {
      EpiTerms none;
      none.count = 0;
      ops.tally(2, 1);
      ops.gemm(n, X, 0.0, Mi, 0.0, 1.0, none, OutView{XMi, 0});
    }
    double nd, nx;
    ops.db_update_product(X, Mk, Mi, XMi, it == 1, mu, imu, mu2, imu2, n, &nd, &nx);
    const double delta = nd / nx;
    if (!(delta == delta)) { status = 2; break; }
    if (delta <= tol || pred <= tol) { status = 0; break; }
    if (!scale && dprev <= 1e-7 && delta > 0.5 * dprev) { status = 0; break; }
    if (delta < 1e-2) scale = 0;
    dprev = delta;
  }
  *iters_out = it > max_db ? max_db : it;
  return status;
}

// Factor coefficients h_{j,i}, g_{j,i} of P_i (i = 2..j+1) in product j >= 2.
static __device__ __forceinline__ void scheme64(int k, int j, int i, double* h, double* g) {
  *h = 0.0;
  *g = 0.0;
  if (k == 2) {
    if (j == 2) {
      *h = (i == 3) ? 1.0 : 0.0;
      *g = (i == 2) ? 1.0 / 3.0 : (i == 3 ? 0.25 : 0.0);
    }
    return;
  }
  if (k == 3) {  // eq. (eqP8pol) in the degree-optimal form
    double c[6];
    k3_coeffs(c);
    if (j == 2) {  // P_4 = P_3 (c3 P_2 + c4 P_3)
      *h = (i == 3) ? 1.0 : 0.0;
      *g = (i == 2) ? c[0] : (i == 3 ? c[1] : 0.0);
    } else if (j == 3) {  // P_5 = (d1 P_2 + d2 P_3 + P_4)(e2 P_3 + P_4)
      *h = (i == 2) ? c[2] : (i == 3 ? c[3] : 1.0);
      *g = (i == 2) ? 0.0 : (i == 3 ? c[4] : 1.0);
    }
    return;
  }
  if (k == 4) {  // the 14+ scheme (c_k4)
    const double* c = c_k4;
    if (j == 2) {  // P_4 = P_3 (c3 P_2 + c4 P_3)
      *h = (i == 3) ? 1.0 : 0.0;
      *g = (i == 2) ? c[0] : (i == 3 ? c[1] : 0.0);
    } else if (j == 3) {  // P_5 = (d1 P_2 + d2 P_3 + P_4)(e2 P_3 + P_4)
      *h = (i == 2) ? c[2] : (i == 3 ? c[3] : 1.0);
      *g = (i == 2) ? 0.0 : (i == 3 ? c[4] : 1.0);
    } else if (j == 4) {  // P_6 = (f1 P_2 + f2 P_3 + f4 P_4 + P_5)(g1 P_2 + g4 P_4 + P_5)
      *h = (i == 2) ? c[5] : (i == 3 ? c[6] : (i == 4 ? c[7] : 1.0));
      *g = (i == 2) ? c[8] : (i == 3 ? 0.0 : (i == 4 ? c[9] : 1.0));
    }
    return;
  }
  int t = 0;
  for (int jj = 2; jj < j; ++jj) t += jj;
  *h = c_h5[t + i - 2];
  *g = c_g5[t + i - 2];
}

static __device__ __forceinline__ double y64(int k, int i) {  // y_i, i = 2..k+2
  if (k == 1) return i == 2 ? 1.0 : 0.5;
  if (k == 2) return i == 2 ? 1.0 : (i == 3 ? 0.5 : 1.0);
  if (k == 3) {
    if (i == 4) {
      double c[6];
      k3_coeffs(c);
      return c[5];
    }
    return i == 2 ? 1.0 : (i == 3 ? 0.5 : 1.0);
  }
  if (k == 4) return i == 2 ? 1.0 : (i == 6 ? 1.0 : c_k4[10 + i - 3]);  // y3, y4, y5 at i = 3, 4, 5
  return c_y5[i - 1];
}

// ---------------------------------------------------------------------------
// Graph evaluation, eq. (five_mult_degopt): out = scale * z(X) with P_2 = X
// (Acur), P_3 = X^2 (A2) given. For Algorithm 1, scale = -2^s (eq. logipASTM
// and the final squaring step): a power of two, so it changes no rounding.
// ---------------------------------------------------------------------------
#if LG_WITH_K6
// k = 6 in the slot's seven matrices. P_2 .. P_6 fill Acur, A2, Y, W1, W2 and
// the factors of P_7 = (sum h_{5,i} P_i)(sum g_{5,i} P_i) take T1, T2. Before
// that product, one elementwise pass replaces P_2 .. P_6 by the three
// combinations of them the rest needs (same element in, same element out, so
// in place): C_L = sum_{i<=6} h_{6,i} P_i, C_R = sum_{i<=6} g_{6,i} P_i and
// C_Y = sum_{i<=6} y_i P_i. Then P_7 goes to W1, the last factors are
// C_L + h_{6,7} P_7 and C_R + g_{6,7} P_7, and the last product's epilogue
// adds scale (C_Y + y_7 P_7): z = y_8 P_8 + sum_{i<=7} y_i P_i.
// Outlined: inlined, its temporaries raised the register pressure of the
// whole execute kernel.
template <class Ops>
static __device__ __noinline__ void graph_eval_k6(Ops& ops, int n, Slot& M, double scale, OutView out) {
  double* P[7] = {nullptr, nullptr, M.Acur, M.A2, M.Y, M.W1, M.W2};
  EpiTerms none;
  none.count = 0;
  int t = 0;  // index of h_{j,2} in c_h6
  for (int j = 2; j <= 5; t += j, ++j) {
    EpiTerms hl, gl;
    hl.count = gl.count = j;
    for (int i = 2; i <= j + 1; ++i) {
      hl.M[i - 2] = gl.M[i - 2] = P[i];
      hl.c[i - 2] = c_h6[t + i - 2];
      gl.c[i - 2] = c_g6[t + i - 2];
    }
    ops.lincomb(n, hl, M.T1);
    ops.lincomb(n, gl, M.T2);
    if (j < 5) {
      ops.tally(2, 1);
      ops.gemm(n, M.T1, 0.0, M.T2, 0.0, 1.0, none, OutView{P[j + 2], 0});
    }
  }
  // t = 14: h_{6,2..7}, g_{6,2..7}
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = ops.tid(); e < nn; e += ops.nthreads()) {
    double v[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = P[i + 2][e];
    double cl = 0.0, cr = 0.0, cy = v[0];  // y_2 = 1
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      cl = fma(c_h6[t + i], v[i], cl);
      cr = fma(c_g6[t + i], v[i], cr);
    }
#pragma unroll
    for (int i = 1; i < 5; ++i) cy = fma(c_y6[i - 1], v[i], cy);
    P[2][e] = cl;
    P[3][e] = cr;
    P[4][e] = cy;
  }
  ops.sync();
  ops.tally(2, 1);
  ops.gemm(n, M.T1, 0.0, M.T2, 0.0, 1.0, none, OutView{M.W1, 0});  // P_7
  EpiTerms l6{{M.Acur, M.W1}, {1.0, c_h6[t + 5]}, 2};
  EpiTerms r6{{M.A2, M.W1}, {1.0, c_g6[t + 5]}, 2};
  ops.lincomb(n, l6, M.W2);
  ops.lincomb(n, r6, M.T1);
  EpiTerms e{{M.Y, M.W1}, {scale, scale * c_y6[4]}, 2};
  ops.tally(2, 1);
  ops.gemm(n, M.W2, 0.0, M.T1, 0.0, scale * c_y6[5], e, out);
}
#endif

template <class Ops>
static __device__ void graph_eval(Ops& ops, int k, int n, Slot& M, double scale, OutView out) {
#if LG_WITH_K6
  if (k == 6) {
    graph_eval_k6(ops, n, M, scale, out);
    return;
  }
#endif
  double* P2 = M.Acur;
  double* P3 = M.A2;
  if (k == 1) {  // z = X + X^2/2 (Taylor T_2)
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) store_out(out, t, scale * fma(0.5, P3[t], P2[t]));
    ops.sync();
    return;
  }
  if (k == 2) {  // P_4 = X^2 (X/3 + X^2/4); z = X + X^2/2 + P_4 (Taylor T_4)
    EpiTerms r{{P2, P3}, {1.0 / 3.0, 0.25}, 2};
    ops.lincomb(n, r, M.T2);
    EpiTerms e{{P2, P3}, {scale, 0.5 * scale}, 2};
    ops.tally(2, 1);
    ops.gemm(n, P3, 0.0, M.T2, 0.0, scale, e, out);
    return;
  }
  if (k == 3) {  // eq. (eqP8pol): P_4 = P_3 (c3 X + c4 P_3), z = (P_4 + d2 P_3 + d1 X)(P_4 + e2 P_3) + ...
    double c[6];
    k3_coeffs(c);
    EpiTerms r{{P2, P3}, {c[0], c[1]}, 2};
    ops.lincomb(n, r, M.T2);
    EpiTerms none;
    none.count = 0;
    ops.tally(2, 1);
    ops.gemm(n, P3, 0.0, M.T2, 0.0, 1.0, none, OutView{M.Y, 0});  // P_4 = y02
    EpiTerms hl{{M.Y, P3, P2}, {1.0, c[3], c[2]}, 3};
    EpiTerms gl{{M.Y, P3}, {1.0, c[4]}, 2};
    ops.lincomb(n, hl, M.T1);
    ops.lincomb(n, gl, M.T2);
    EpiTerms e{{M.Y, P3, P2}, {scale * c[5], 0.5 * scale, scale}, 3};
    ops.tally(2, 1);
    ops.gemm(n, M.T1, 0.0, M.T2, 0.0, scale, e, out);
    return;
  }
  // k = 4 (the 14+ scheme, P_4 .. P_6) and k = 5 (Table table_simple_experiment,
  // P_4 .. P_7): factors from scheme64, the last product's epilogue adds
  // sum_{i <= k+1} y_i P_i and scales
  double* P[8] = {nullptr, nullptr, P2, P3, M.Y, M.W1, M.W2, nullptr};
  for (int j = 2; j <= k; ++j) {
    EpiTerms hl, gl;
    hl.count = gl.count = j;
    for (int i = 2; i <= j + 1; ++i) {
      double h, g;
      scheme64(k, j, i, &h, &g);
      hl.M[i - 2] = P[i];
      hl.c[i - 2] = h;
      gl.M[i - 2] = P[i];
      gl.c[i - 2] = g;
    }
    ops.lincomb(n, hl, M.T1);
    ops.lincomb(n, gl, M.T2);
    ops.tally(2, 1);
    if (j < k) {
      EpiTerms none;
      none.count = 0;
      ops.gemm(n, M.T1, 0.0, M.T2, 0.0, 1.0, none, OutView{P[j + 2], 0});
    } else {
      EpiTerms e;
      e.count = k;
      for (int i = 2; i <= k + 1; ++i) {
        e.M[i - 2] = P[i];
        e.c[i - 2] = scale * y64(k, i);
      }
      ops.gemm(n, M.T1, 0.0, M.T2, 0.0, scale * y64(k, k + 2), e, out);
    }
  }
}

// ---------------------------------------------------------------------------
// Balancing, the optional preprocessing A <- T^{-1} A T of Algorithm 1 (Step
// 1) and the postprocessing L <- T L T^{-1}: T diagonal with powers of two
// (radix-2 Parlett-Reinsch). For each i in turn, c and r are the 1-norms of
// the off-diagonal parts of column i and row i; the power of two f that
// brings c f and r / f within a factor 2 of each other is applied (column i
// times f, row i divided by f) when it cuts c + r by more than 5 %. Sweeps
// repeat until one applies nothing (at most 100). Zero rows or columns are
// left alone. Every factor is a power of two, so both similarities are exact.
// d (global, n doubles) gets diag(T).
// ---------------------------------------------------------------------------
template <class Ops>
static __device__ void balance_matrix(Ops& ops, double* A, int n, double* d) {
  for (int i = ops.tid(); i < n; i += ops.nthreads()) d[i] = 1.0;
  ops.sync();
  for (int sweep = 0; sweep < 100; ++sweep) {
    int changed = 0;
    for (int i = 0; i < n; ++i) {
      double c = 0.0, r = 0.0;
      for (int j = ops.tid(); j < n; j += ops.nthreads())
        if (j != i) {
          c += fabs(A[(int64_t)j * n + i]);
          r += fabs(A[(int64_t)i * n + j]);
        }
      c = ops.sum(c);
      r = ops.sum(r);
      if (c == 0.0 || r == 0.0) continue;
      const double s = c + r;
      double f = 1.0, g = r * 0.5;
      while (c < g) {
        f *= 2.0;
        c *= 4.0;
      }
      g = r * 2.0;
      while (c >= g) {
        f *= 0.5;
        c *= 0.25;
      }
      if ((c + r) / f < 0.95 * s) {
        changed = 1;
        const double fi = 1.0 / f;  // a power of two: exact
        for (int j = ops.tid(); j < n; j += ops.nthreads()) {
          A[(int64_t)i * n + j] *= fi;
          A[(int64_t)j * n + i] *= f;
        }
        if (ops.leader()) d[i] *= f;
        ops.sync();
      }
    }
    if (!changed) break;
  }
}

// M_ij <- M_ij d_i / d_j (T M T^{-1}) or, with inverse, M_ij d_j / d_i
// (T^{-1} M T), for an FP64 work matrix.
template <class Ops>
static __device__ void similarity_diag(Ops& ops, double* Mx, int n, const double* d, bool inverse) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) {
    const int i = (int)(t / n), j = (int)(t % n);
    Mx[t] *= inverse ? d[j] / d[i] : d[i] / d[j];
  }
  ops.sync();
}

// The output L <- T L T^{-1} in place, in the caller's dtype.
template <class Ops>
static __device__ void unbalance_output(Ops& ops, void* L, int dtype, int64_t off, int n, const double* d) {
  ops.sync();
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) {
    const double f = d[t / n] / d[t % n];
    if (dtype == 0) {
      static_cast<double*>(L)[off + t] *= f;
    } else {
      float* q = static_cast<float*>(L) + off + t;
      *q = (float)((double)*q * f);
    }
  }
  ops.sync();
}

// ---------------------------------------------------------------------------
// One matrix, per entry point.
// ---------------------------------------------------------------------------
template <class Ops>
static __device__ void run_execute(Ops& ops, const SmallParams& p, int b, int n, int64_t off, Slot& M) {
  const int km = p.k_max;
  ops.tally_reset();
  const int finite = load_matrix(ops, p.A, p.dtype, off, n, M.Acur);
  if (!finite) {
    fill_nan(ops, p.L, p.dtype, off, n);
    if (ops.leader()) {
      if (p.stats)
        for (int t = 0; t < 4; ++t) p.stats[4 * b + t] = 0;
      p.info[b] = 4;
      if (p.s_out) p.s_out[b] = 0;
      if (p.k_out) p.k_out[b] = km;
    }
    return;
  }
  double* dvec = p.balance ? p.bal + (int64_t)b * p.bal_stride : nullptr;
  if (dvec) balance_matrix(ops, M.Acur, n, dvec);
  const int m = LG_M_OF(km);
  const double th = LG_THETA(p.theta, km);
  double nB = ops.norm1(M.Acur, n, 1.0), nI2 = 0.0;
  int s = 0, have_ai2 = 0, info = 0, finish = nB <= th;
  double alpha = nB;
  EstState last{-1.0, -1.0, m, 0};
  int reuse = 0;          // the previous level's Y can replace the next first inversion
  double ld_carry = 0.0;  // log|det| of the next level's A
  while (!finish && s < p.max_sqrt) {
    EstState st{-1.0, -1.0, m, 0};
    finish = alpha_test(ops, M.Acur, have_ai2 ? M.A2 : nullptr, n, nB, nI2, m, th, st, &alpha);
    last = st;
    if (finish) break;
    if (p.ctx && s < p.ctx_levels) {
      double* ck = p.ctx + ((int64_t)b * p.ctx_levels + s) * (int64_t)p.ctx_nmax * p.ctx_nmax;
      copy_matrix(ops, ck, M.Acur, n);
    }
    copy_matrix(ops, M.A2, M.Acur, n);
    int it;
    const int r = p.db_form == 1 ? db_sqrt_product(ops, M, n, p.max_db, &it)
                                 : db_sqrt(ops, M, n, p.max_db, &it, nullptr, reuse, &ld_carry);
    reuse = p.db_form != 1 && r == 0;
    if (r == 1) { info = 1; break; }
    if (r == 2 && info == 0) info = 2;
    ai2_from(ops, M, n);
    nB = ops.norm1(M.Acur, n, 1.0);
    nI2 = ops.norm1(M.A2, n, 0.0);
    have_ai2 = 1;
    ++s;
  }
  int k = km;
  if (info == 1) {
    fill_nan(ops, p.L, p.dtype, off, n);
  } else {
    if (!finish && info == 0) info = 3;
    if (!have_ai2) {
      EpiTerms none;
      none.count = 0;
      ops.tally(2, 1);
      ops.gemm(n, M.Acur, 1.0, M.Acur, 1.0, 1.0, none, OutView{M.A2, 0});
      nI2 = ops.norm1(M.A2, n, 0.0);
    }
    if (finish) k = order_search(ops, M.Acur, M.A2, n, nB, nI2, km, p.theta, last.t_m >= 0.0 ? &last : nullptr);
    to_x(ops, M.Acur, n);  // P_2 = X = -(A - I)
    if (p.gbuf) {
      // precision form: P_2 and P_3 go to the tensor-core graph stage in FP32
      float* g = p.gbuf + (int64_t)b * 5 * (int64_t)p.gbuf_nmax * p.gbuf_nmax;
      float* g3 = g + (int64_t)p.gbuf_nmax * p.gbuf_nmax;
      const int64_t nn = (int64_t)n * n;
      for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) {
        g[t] = static_cast<float>(M.Acur[t]);
        g3[t] = static_cast<float>(M.A2[t]);
      }
      ops.sync();
    } else {
      graph_eval(ops, k, n, M, -ldexp(1.0, s), out_view(p.L, p.dtype, off));
      if (dvec) unbalance_output(ops, p.L, p.dtype, off, n, dvec);
    }
  }
  if (ops.leader()) {
    p.info[b] = info;
    if (p.s_out) p.s_out[b] = s;
    if (p.k_out) p.k_out[b] = k;
    if (p.ctx_hdr) {
      p.ctx_hdr[2 * b] = s;
      p.ctx_hdr[2 * b + 1] = (info == 0 || info == 2 || info == 3) ? k : -1;
    }
    if (p.alpha) p.alpha[b] = alpha;
    if (p.stats)
      for (int t = 0; t < 4; ++t) p.stats[4 * b + t] = ops.tally_get(t);
  }
}

template <class Ops>
static __device__ void run_plan(Ops& ops, const SmallParams& p, int b, int n, int64_t off, Slot& M) {
  const int km = p.k_max;
  const int finite = load_matrix(ops, p.A, p.dtype, off, n, M.Acur);
  int fin2 = 1;
  if (p.AI2_in) fin2 = load_matrix(ops, p.AI2_in, p.dtype, off, n, M.A2);
  if (!finite || !fin2) {
    if (ops.leader()) {
      p.info[b] = 4;
      p.finish[b] = 0;
      p.k_out[b] = km;
      p.alpha[b] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  const int m = LG_M_OF(km);
  const double th = LG_THETA(p.theta, km);
  const double nB = ops.norm1(M.Acur, n, 1.0);
  EstState st{-1.0, -1.0, m, 0};
  int fin;
  double a;
  double nI2 = p.AI2_in ? ops.norm1(M.A2, n, 0.0) : 0.0;
  if (!p.AI2_in && nB <= th) {
    fin = 1;
    a = nB;
  } else {
    fin = alpha_test(ops, M.Acur, p.AI2_in ? M.A2 : nullptr, n, nB, nI2, m, th, st, &a);
  }
  if (!p.AI2_in) {
    EpiTerms none;
    none.count = 0;
    ops.gemm(n, M.Acur, 1.0, M.Acur, 1.0, 1.0, none, OutView{M.A2, 0});
    nI2 = ops.norm1(M.A2, n, 0.0);
  }
  const int k = fin ? order_search(ops, M.Acur, M.A2, n, nB, nI2, km, p.theta, &st) : km;
  if (ops.leader()) {
    p.info[b] = 0;
    p.finish[b] = fin;
    p.k_out[b] = k;
    p.alpha[b] = a;
  }
}

template <class Ops>
static __device__ void run_sqrt(Ops& ops, const SmallParams& p, int b, int n, int64_t off, Slot& M) {
  const int finite = load_matrix(ops, p.A_inout, p.dtype, off, n, M.Acur);
  if (!finite) {
    if (ops.leader()) {
      p.info[b] = 4;
      if (p.iters) p.iters[b] = 0;
    }
    return;
  }
  copy_matrix(ops, M.A2, M.Acur, n);
  if (p.A2_out) store_matrix(ops, p.A2_out, p.dtype, off, n, M.A2);
  int it;
  const int r = p.db_form == 1 ? db_sqrt_product(ops, M, n, p.max_db, &it) : db_sqrt(ops, M, n, p.max_db, &it);
  store_matrix(ops, p.A_inout, p.dtype, off, n, M.Acur);
  if (p.AI2_out) {
    ai2_from(ops, M, n);
    store_matrix(ops, p.AI2_out, p.dtype, off, n, M.A2);
  }
  if (ops.leader()) {
    p.info[b] = r;
    if (p.iters) p.iters[b] = it;
  }
}

template <class Ops>
static __device__ void run_graph(Ops& ops, const SmallParams& p, int b, int n, int64_t off, Slot& M) {
  const int k = p.k_in[b];
  if (!(k >= 1 && k <= LG_MAX_ORDER)) {
    if (ops.leader() && p.info) p.info[b] = -1;
    return;
  }
  load_matrix(ops, p.X, p.dtype, off, n, M.Acur);
  if (p.P3) {
    load_matrix(ops, p.P3, p.dtype, off, n, M.A2);
  } else {
    EpiTerms none;
    none.count = 0;
    ops.gemm(n, M.Acur, 0.0, M.Acur, 0.0, 1.0, none, OutView{M.A2, 0});
  }
  graph_eval(ops, k, n, M, 1.0, out_view(p.L, p.dtype, off));
  if (ops.leader() && p.info) p.info[b] = 0;
}

// ---------------------------------------------------------------------------
// Adjoint (differentiation form): dA = gradient of sum(dL o L) for the map
// A -> L that the forward computed, at the forward's plan (s, k). Reverse
// mode through the graph products (P = L_j R_j gives Lbar = Pbar R_j^T and
// Rbar = L_j^T Pbar, scattered to the P_i by h_{j,i} and g_{j,i}), through
// A_I2 = A_2 - 2A + I, X = I - A, and through every Denman-Beavers iteration
// (Xbar_i = mu/2 Xbar_{i+1} - 1/(2 mu) X_i^{-T} Ybar_{i+1} X_i^{-T}, and the
// same with X, Y exchanged) with mu_i held fixed: its derivative does not
// change the converged root. A level's iterates are recomputed from the
// level's input, which the forward checkpointed.
// ---------------------------------------------------------------------------
struct BwdSlot {
  Slot F;          // forward recompute: Acur/P_2, A2/P_3, Y/P_4, W1/P_5, W2/P_6, T1, T2
  double* Pb[6];   // adjoints of P_2 .. P_7
  double *Lb, *Rb, *Ab, *Yb;
  DbTape tape;
};

template <class Ops>
static __device__ void factor_terms(int k, int j, double* const* P, EpiTerms& hl, EpiTerms& gl) {
  hl.count = gl.count = j;
  for (int i = 2; i <= j + 1; ++i) {
    double h, g;
    scheme64(k, j, i, &h, &g);
    hl.M[i - 2] = gl.M[i - 2] = P[i];
    hl.c[i - 2] = h;
    gl.c[i - 2] = g;
  }
}

template <class Ops>
static __device__ void run_backward(Ops& ops, const SmallParams& p, int b, int n, int64_t off, BwdSlot& W) {
  const int s = p.ctx_hdr[2 * b], k = p.ctx_hdr[2 * b + 1];
  const int64_t nn = (int64_t)n * n;
  if (k < 1 || k > 5) {  // the forward produced no result
    fill_nan(ops, p.dA, p.dtype, off, n);
    if (ops.leader()) p.info[b] = 1;
    return;
  }
  if (s > p.ctx_levels) {  // the forward could not checkpoint every level
    fill_nan(ops, p.dA, p.dtype, off, n);
    if (ops.leader()) p.info[b] = 6;
    return;
  }
  const int64_t lstride = (int64_t)p.ctx_nmax * p.ctx_nmax;
  const double* dvec = p.balance ? p.bal + (int64_t)b * p.bal_stride : nullptr;
  Slot& F = W.F;
  int it = 0, status = 0;
  // 1. recompute the last level (its tape serves the first reversal) and P_3
  if (s >= 1) {
    copy_matrix(ops, F.Acur, p.ctx + ((int64_t)b * p.ctx_levels + (s - 1)) * lstride, n);
    copy_matrix(ops, F.A2, F.Acur, n);
    if (db_sqrt(ops, F, n, p.max_db, &it, &W.tape) == 1) status = 1;
    ai2_from(ops, F, n);
  } else {
    load_matrix(ops, p.A, p.dtype, off, n, F.Acur);
    if (dvec) similarity_diag(ops, F.Acur, n, dvec, true);  // T^{-1} A T
    EpiTerms none;
    none.count = 0;
    ops.gemm(n, F.Acur, 1.0, F.Acur, 1.0, 1.0, none, OutView{F.A2, 0});
  }
  to_x(ops, F.Acur, n);
  double* P[7] = {nullptr, nullptr, F.Acur, F.A2, F.Y, F.W1, F.W2};
  // 2. recompute the products that later products use as factors
  const int last_j = k;  // P_{k+2} is the last product
  for (int j = 2; j < last_j; ++j) {
    EpiTerms hl, gl;
    factor_terms<Ops>(k, j, P, hl, gl);
    ops.lincomb(n, hl, F.T1);
    ops.lincomb(n, gl, F.T2);
    EpiTerms none;
    none.count = 0;
    ops.gemm(n, F.T1, 0.0, F.T2, 0.0, 1.0, none, OutView{P[j + 2], 0});
  }
  // 3. zbar = -2^s dL; Pbar_i = y_i zbar
  load_matrix(ops, p.dL, p.dtype, off, n, W.Lb);
  if (dvec) similarity_diag(ops, W.Lb, n, dvec, false);  // the adjoint of L = T z T^{-1}: T Lbar T^{-1}
  const double sc = -ldexp(1.0, s);
  for (int i = 2; i <= k + 2; ++i) {
    EpiTerms e{{W.Lb}, {sc * y64(k, i)}, 1};
    ops.lincomb(n, e, W.Pb[i - 2]);
  }
  // 4. reverse the products, last first
  for (int j = last_j; j >= 2; --j) {
    EpiTerms hl, gl;
    factor_terms<Ops>(k, j, P, hl, gl);
    ops.lincomb(n, hl, F.T1);  // L_j
    ops.lincomb(n, gl, F.T2);  // R_j
    EpiTerms none;
    none.count = 0;
    ops.gemm(n, W.Pb[j], 0.0, F.T2, 0.0, 1.0, none, OutView{W.Lb, 0}, false, true);  // Lbar = Pbar R^T
    ops.gemm(n, F.T1, 0.0, W.Pb[j], 0.0, 1.0, none, OutView{W.Rb, 0}, true, false);  // Rbar = L^T Pbar
    for (int i = 2; i <= j + 1; ++i) {
      EpiTerms u{{W.Pb[i - 2], W.Lb, W.Rb}, {1.0, hl.c[i - 2], gl.c[i - 2]}, 3};
      ops.lincomb(n, u, W.Pb[i - 2]);
    }
  }
  // 5. P_3: X X when s = 0, else A_2 - 2A + I
  double* Xb = W.Pb[0];
  if (s == 0) {
    EpiTerms acc{{Xb}, {1.0}, 1};
    ops.gemm(n, W.Pb[1], 0.0, F.Acur, 0.0, 1.0, acc, OutView{Xb, 0}, false, true);  // += P3bar X^T
    ops.gemm(n, F.Acur, 0.0, W.Pb[1], 0.0, 1.0, acc, OutView{Xb, 0}, true, false);  // += X^T P3bar
  }
  {  // Abar_s = -Xbar (- 2 P3bar when P_3 = A_I2)
    EpiTerms e{{Xb, W.Pb[1]}, {-1.0, s >= 1 ? -2.0 : 0.0}, 2};
    ops.lincomb(n, e, W.Ab);
  }
  // 6. reverse the square-root levels, last first
  for (int lev = s - 1; lev >= 0 && !status; --lev) {
    if (lev < s - 1) {
      copy_matrix(ops, F.Acur, p.ctx + ((int64_t)b * p.ctx_levels + lev) * lstride, n);
      if (db_sqrt(ops, F, n, p.max_db, &it, &W.tape) == 1) status = 1;
    }
    if (status) break;
    if (it > W.tape.cap) {
      status = 2;
      break;
    }
    for (int64_t t = ops.tid(); t < nn; t += ops.nthreads()) W.Yb[t] = 0.0;
    ops.sync();
    for (int i = it - 1; i >= 0; --i) {
      const double* Xi = W.tape.inv + (int64_t)(2 * i) * W.tape.stride;
      const double* Yi = W.tape.inv + (int64_t)(2 * i + 1) * W.tape.stride;
      const double mu = W.tape.mu[i];
      EpiTerms none;
      none.count = 0;
      ops.gemm(n, Xi, 0.0, W.Yb, 0.0, 1.0, none, OutView{W.Lb, 0}, true, false);  // X_i^{-T} Ybar
      if (i > 0) ops.gemm(n, Yi, 0.0, W.Ab, 0.0, 1.0, none, OutView{W.Rb, 0}, true, false);  // Y_i^{-T} Xbar
      EpiTerms ex{{W.Ab}, {0.5 * mu}, 1};
      ops.gemm(n, W.Lb, 0.0, Xi, 0.0, -0.5 / mu, ex, OutView{W.Ab, 0}, false, true);
      if (i > 0) {
        EpiTerms ey{{W.Yb}, {0.5 * mu}, 1};
        ops.gemm(n, W.Rb, 0.0, Yi, 0.0, -0.5 / mu, ey, OutView{W.Yb, 0}, false, true);
      }
    }
    if (lev == s - 1) {  // the A_2 term of A_I2 = A_2 - 2A + I
      EpiTerms e{{W.Ab, W.Pb[1]}, {1.0, 1.0}, 2};
      ops.lincomb(n, e, W.Ab);
    }
  }
  if (status) {
    fill_nan(ops, p.dA, p.dtype, off, n);
    if (ops.leader()) p.info[b] = status == 1 ? 1 : 6;
    return;
  }
  if (dvec) similarity_diag(ops, W.Ab, n, dvec, true);  // the adjoint of T^{-1} A T: T^{-1} Abar T
  store_matrix(ops, p.dA, p.dtype, off, n, W.Ab);
  if (ops.leader()) p.info[b] = 0;
}

}  // namespace LG_NS
