// scheme_f32.cuh -- the graph schemes of the degree-optimal form (Sec. 3,
// eq. five_mult_degopt) in FP32, for the split-precision product kernels
// (graph_tc.cu, graph_tma.cu). The FP64 path has its own tables in
// logm_algo.cuh.
#pragma once

#include <cstdint>

namespace lg {

// Scheme tables (Sec. 3): index j = product number (1: P_3 = X X, 2..5), terms
// i = 2..j+1 of the factors, y_i of the output. Table table_simple_experiment
// for k = 5; exact Taylor T_4 (eq. Taylor_log) for k = 2; T_8 by eq.
// (eqP8pol) for k = 3, its coefficients solved in closed form below; the 14+
// scheme for k = 4.
static __constant__ float c_tc_h5[14] = {
    7.363757032799957e-02f, -1.050281301619960e+00f, 8.897468955192446e-02f,
    -1.599651928992725e-01f, 9.577281350989334e-01f, 5.394999133948797e-01f,
    6.700731102561937e-02f, -5.158769100223212e-02f, 1.094308587350110e+00f,
    1.027072285939197e-01f, -8.964023050065877e-03f, -2.100705663612491e-01f,
    1.949655359168707e-01f, 1.117368056772713e+00f};
static __constant__ float c_tc_g5[14] = {
    -9.666134174379001e-01f, -4.395519034717933e-01f, 1.048664069004776e-01f,
    1.585606124033259e-01f, 1.668066506920988e-01f, -8.025600931705978e-02f,
    -1.159854366397558e-01f, 1.066554944706011e-01f, 1.127094008297975e+00f,
    2.702180425508705e-01f, 4.137541209720699e-02f, 4.857347452405025e-01f,
    -6.000256005636980e-01f, 1.063393233943084e+00f};
static __constant__ float c_tc_y5[7] = {0.0f, 1.0f, 5.065546620208965e-01f, 3.832512052972577e-01f,
                                        1.088307723749078e+00f, 2.787461897212877e-01f,
                                        8.157421998489228e-01f};

// k = 4, the 14+ scheme of Sec. 3 (degree 16, T_14 matched; the paper prints
// no coefficients): the real root of "coefficient of x^i = 1/i, i = 2..14"
// with the smallest coefficients. P_4 = P_3 (c3 X + c4 P_3), P_5 = (d1 X +
// d2 P_3 + P_4)(e2 P_3 + P_4), P_6 = (f1 X + f2 P_3 + f4 P_4 + P_5)(g1 X +
// g4 P_4 + P_5), z = X + y3 P_3 + y4 P_4 + y5 P_5 + P_6.
// Order: c3 c4 d1 d2 e2 f1 f2 f4 g1 g4 y3 y4 y5.
static __constant__ float c_tc_k4[13] = {
    0.3602750956560524f,  0.3018442985303789f,   0.3412287952056341f,  -0.18047064940974122f,
    0.18907274365286242f, -0.014079460349863975f, 0.24400741065645315f, -0.8525627910338015f,
    0.1463535711919622f,  0.9787518426666669f,   0.5020605793026582f,  0.6095606808527384f,
    1.2091753609836204f};

struct Coeffs {
  float h[6], g[6];  // factor coefficients for P_2 .. P_{j+1}
  int terms;         // j (number of P_i in each factor)
};

// k = 3, eq. (eqP8pol): y02 = X^2 (c4 X^2 + c3 X), z = (y02 + d2 X^2 + d1 X)
// (y02 + e2 X^2) + e0 y02 + X^2/2 + X. Matching x^8 .. x^3 with 1/8 .. 1/3
// gives c4 = 1/sqrt(8), c3 = 1/(14 c4), d2 + e2 = S, d1, and a quadratic in
// e2 whose root with the smaller coefficients is taken. Solved in FP64, used
// in FP32. c = c3, c4, d1, d2, e2, e0.
static __device__ __forceinline__ void tc_k3_coeffs(float* c) {
  const double c4 = 1.0 / sqrt(8.0);
  const double c3 = 1.0 / (14.0 * c4);
  const double sum = (1.0 / 6.0 - c3 * c3) / c4;
  const double d1 = (1.0 / 5.0 - c3 * sum) / c4;
  const double beta = sum - c4 * d1 / c3;
  const double gamma = c3 * d1 + c4 / (3.0 * c3) - 0.25;
  const double e2 = 0.5 * (beta + sqrt(beta * beta + 4.0 * gamma));
  c[0] = (float)c3;
  c[1] = (float)c4;
  c[2] = (float)d1;
  c[3] = (float)(sum - e2);
  c[4] = (float)e2;
  c[5] = (float)((1.0 / 3.0 - d1 * e2) / c3);
}

// Factor coefficients of product j for a matrix evaluated with k products.
static __device__ __forceinline__ void scheme_coeffs(int k, int j, Coeffs& c) {
  for (int t = 0; t < 6; ++t) c.h[t] = c.g[t] = 0.0f;
  if (j == 1) {  // P_3 = X X (Theorem of Sec. 3: h_{1,2} = g_{1,2} = 1)
    c.terms = 1;
    c.h[0] = c.g[0] = 1.0f;
    return;
  }
  c.terms = j;
  if (k == 2) {  // P_4 = P_3 (X/3 + P_3/4)
    c.h[1] = 1.0f;
    c.g[0] = 1.0f / 3.0f;
    c.g[1] = 0.25f;
    return;
  }
  if (k == 3) {
    float q[6];
    tc_k3_coeffs(q);
    if (j == 2) {  // P_4 = P_3 (c3 X + c4 P_3)
      c.h[1] = 1.0f;
      c.g[0] = q[0];
      c.g[1] = q[1];
    } else {  // P_5 = (d1 X + d2 P_3 + P_4)(e2 P_3 + P_4)
      c.h[0] = q[2];
      c.h[1] = q[3];
      c.h[2] = 1.0f;
      c.g[1] = q[4];
      c.g[2] = 1.0f;
    }
    return;
  }
  if (k == 4) {
    const float* q = c_tc_k4;
    if (j == 2) {  // P_4 = P_3 (c3 X + c4 P_3)
      c.h[1] = 1.0f;
      c.g[0] = q[0];
      c.g[1] = q[1];
    } else if (j == 3) {  // P_5 = (d1 X + d2 P_3 + P_4)(e2 P_3 + P_4)
      c.h[0] = q[2];
      c.h[1] = q[3];
      c.h[2] = 1.0f;
      c.g[1] = q[4];
      c.g[2] = 1.0f;
    } else {  // P_6 = (f1 X + f2 P_3 + f4 P_4 + P_5)(g1 X + g4 P_4 + P_5)
      c.h[0] = q[5];
      c.h[1] = q[6];
      c.h[2] = q[7];
      c.h[3] = 1.0f;
      c.g[0] = q[8];
      c.g[2] = q[9];
      c.g[3] = 1.0f;
    }
    return;
  }
  int t = 0;
  for (int jj = 2; jj < j; ++jj) t += jj;
  for (int i = 0; i < j; ++i) {
    c.h[i] = c_tc_h5[t + i];
    c.g[i] = c_tc_g5[t + i];
  }
}

// y_2 .. y_{k+2} of the scheme (index 0 = y_2).
static __device__ __forceinline__ float scheme_y(int k, int i2) {
  if (k == 1) return i2 == 0 ? 1.0f : (i2 == 1 ? 0.5f : 0.0f);
  if (k == 2) return i2 == 0 ? 1.0f : (i2 == 1 ? 0.5f : (i2 == 2 ? 1.0f : 0.0f));
  if (k == 3) {
    if (i2 == 2) {
      float q[6];
      tc_k3_coeffs(q);
      return q[5];  // e0
    }
    return i2 == 0 ? 1.0f : (i2 == 1 ? 0.5f : (i2 == 3 ? 1.0f : 0.0f));
  }
  if (k == 4) return (i2 == 0 || i2 == 4) ? 1.0f : c_tc_k4[10 + i2 - 1];  // y3, y4, y5 at i2 = 1, 2, 3
  return c_tc_y5[i2 + 1];
}

static __device__ __forceinline__ int needs_product(int k, int p3_given, int j) {
  if (j == 1) return !p3_given;    // P_3 = X X only when the caller did not supply it
  if (k == 2) return j == 2;
  if (k == 3) return j <= 3;
  if (k == 4) return j <= 4;
  if (k == 5) return j <= 5;
  return 0;
}

static __device__ __forceinline__ int is_last_product(int k, int j) {
  return k >= 2 && k <= 5 && j == k;
}

}  // namespace lg
