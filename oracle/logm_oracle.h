/*
 * logm_oracle.h -- interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only code allowed to load this library. The CUDA
 * library never includes this header and this header includes nothing of it.
 *
 * All matrices are dense, row-major, n x n, IEEE binary64.
 */
#ifndef LOGM_ORACLE_H
#define LOGM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-matrix status codes (same meanings as the library's, written here on
 * their own). */
enum {
  ORC_OK = 0,
  ORC_SINGULAR = 1,       /* exact zero pivot in an LU factorisation */
  ORC_NO_CONVERGENCE = 2, /* Denman-Beavers iteration hit its cap */
  ORC_MAX_SQRT = 3,       /* square-root count hit maxiter (Algorithm 1) */
  ORC_NONFINITE = 4       /* NaN or Inf in the input */
};

typedef struct {
  int32_t k_max;       /* largest number of graph products: 1..6 */
  int32_t max_sqrt;    /* maxiter of Algorithm 1 */
  int32_t max_db_iter; /* cap on Denman-Beavers iterations per square root */
  int32_t force_s;     /* < 0: choose s by the bound; >= 0: take exactly s roots */
  int32_t force_k;     /* <= 0: order search; else evaluate with this k */
  int32_t db_form;     /* 0: eq. (ScalDB), two inversions; 1: product form */
  int32_t balance;     /* 0: T = I; 1: diagonal balancing (Algorithm 1, Step 1) */
  int32_t reuse_root;  /* 0: eq. (ScalDB) as written at every level; 1: later levels
                          start from the previous level's Y as A^{-1} (opt-in) */
  double theta[6];     /* Theta_{m_k} for k = 1..6 (Table Table_theta) */
} orc_opts;

typedef struct {
  int32_t s;              /* square roots taken */
  int32_t k;              /* graph products used (1..6) */
  int32_t info;           /* ORC_* status */
  int32_t db_iters;       /* total Denman-Beavers iterations over all levels */
  int32_t n_estimates;    /* calls of the 1-norm power estimator */
  int32_t n_inv;          /* matrix inversions performed by the square roots */
  double alpha;           /* alpha_{m_kmax} value of the pass that set finish */
  double norm_b;          /* ||A^{1/2^s} - I||_1 on exit */
  double norm_ai2;        /* ||(A^{1/2^s} - I)^2||_1 on exit */
  double margin;          /* smallest |x - t| / t over the plan's comparisons x <= t */
  int32_t margin_s;       /* square-root level of that comparison (-1: none made) */
  int32_t reserved;
} orc_diag;

int orc_version(void);

/* Table table_simple_experiment (Sec. 3), exported for the transcription
 * test: h[14] = h_{2,2..3}, h_{3,2..4}, h_{4,2..5}, h_{5,2..6}; g the same;
 * y[7] = y_1..y_7. */
void orc_coeffs_k5(double* h, double* g, double* y);

/* k = 3 coefficients of eq. (eqP8pol), solved in closed form:
 * c[6] = c3, c4, d1, d2, e2, e0. */
void orc_coeffs_k3(double* c);

/* k = 4 coefficients of the 14+ scheme (solved here, see logm_oracle.c):
 * c[13] = c3, c4, d1, d2, e2, f1, f2, f4, g1, g4, y3, y4, y5. */
void orc_coeffs_k4(double* c);

/* k = 6 coefficients (derived here: the paper prints none for k >= 6, see
 * logm_oracle.c): h[20] = h_{2,2..3}, h_{3,2..4}, h_{4,2..5}, h_{5,2..6},
 * h_{6,2..7}; g the same; y[8] = y_1..y_8. */
void orc_coeffs_k6(double* h, double* g, double* y);

void orc_gemm(int n, const double* A, const double* B, double* C);
double orc_norm1(int n, const double* A);
int orc_lu(int n, double* LU, int32_t* piv);
int orc_inverse(int n, const double* A, double* Ainv, double* logabsdet);
int orc_sqrtm_db(int n, const double* A, double* X, int max_iter, int32_t* iters);
int orc_sqrtm_db_product(int n, const double* A, double* X, int max_iter, int32_t* iters);
/* eq. (ScalDB) with a known A^{-1} and log|det A| for the first step. */
int orc_sqrtm_db_reuse(int n, const double* A, double* X, int max_iter, int32_t* iters, const double* Ainv,
                       double logabsdet);
void orc_balance(int n, double* A, double* d);
double orc_normest_pow(int n, const double* B, const double* AI2, int p);
int orc_graph_eval(int n, int k, const double* X, const double* P3, double* Z);
void orc_horner(int n, int deg, const double* b, const double* X, double* Z);
int orc_plan(int n, const double* A, const double* AI2, const orc_opts* o,
             int32_t* finish, int32_t* k, double* alpha);
int orc_logm(int n, const double* A, double* L, const orc_opts* o, orc_diag* d);
int orc_logm_batch(int count, const int32_t* n, const int64_t* offset,
                   const double* A, double* L, const orc_opts* o,
                   orc_diag* d, int nthreads);
void orc_expm_taylor(int n, const double* A, double* E);
int orc_frechet_adjoint(int n, const double* A, const double* W, double* G,
                        const orc_opts* o);

#ifdef __cplusplus
}
#endif
#endif
