// CPU harness for the digit split and level combination of the tensor-core
// FP64 products (paper_2401_10089_gb300/csrc/fp64_slices.cuh): the same
// __host__ __device__ code, compiled for the host by the CPU tests.
#include "../../paper_2401_10089_gb300/csrc/fp64_slices.cuh"

extern "C" {

// Row split: e and kSlices digits for each of k values (digits[i * k + t]).
int32_t h_split(const double* u, int k, int32_t* digits) {
  double m = 0.0;
  for (int t = 0; t < k; ++t) {
    const double a = std::fabs(u[t]);
    if (!(a <= m)) m = a;
  }
  const int32_t e = lg::slice_exponent(m);
  for (int t = 0; t < k; ++t) {
    int32_t d[lg::kSlices];
    if (e == lg::kSliceNonFinite) {
      for (int i = 0; i < lg::kSlices; ++i) d[i] = 0;
    } else {
      lg::slice_digits(lg::slice_fixed(u[t], e), d);
    }
    for (int i = 0; i < lg::kSlices; ++i) digits[i * k + t] = d[i];
  }
  return e;
}

// u.v as the tensor-core path forms it: digit products summed per level in
// exact integers (what the FP32 accumulators hold), passed through the FP32
// representation, combined.
double h_sliced_dot(const double* u, const double* v, int k) {
  int32_t du[lg::kSlices * lg::kSliceK], dv[lg::kSlices * lg::kSliceK];
  const int32_t eu = h_split(u, k, du), ev = h_split(v, k, dv);
  int32_t c[lg::kSliceLevels];
  for (int L = 2; L <= lg::kSlices + 1; ++L) {
    int64_t acc = 0;
    for (int i = 1; i < L; ++i) {
      const int j = L - i;
      if (i > lg::kSlices || j > lg::kSlices) continue;
      for (int t = 0; t < k; ++t) acc += (int64_t)du[(i - 1) * k + t] * dv[(j - 1) * k + t];
    }
    const float f = static_cast<float>(acc);  // exact while |acc| <= 2^24
    c[L - 2] = lg::level_int(f);
  }
  return lg::combine_levels(c, eu, ev);
}

int32_t h_level_int(float v) { return lg::level_int(v); }
int32_t h_level_int_wide(float v) { return lg::level_int_wide(v); }
double h_combine_fp(const int32_t* c, int32_t eu, int32_t ev) { return lg::combine_levels_fp(c, eu, ev); }
double h_combine_fast(const int32_t* c, int32_t eu, int32_t ev, int32_t* slow) {
  bool sl = false;
  const double r = lg::combine_levels_fast(c, eu, ev, &sl);
  *slow = sl ? 1 : 0;
  return r;
}
double h_exact_int_to_double(int64_t x) { return lg::exact_int_to_double(x); }

// the integer-only split against the FP64-scaled one: fixed-point integers
// and digits, 1 when identical
int h_split_routes_agree(double u, int32_t e) {
  const int64_t a = lg::slice_fixed(u, e), b = lg::slice_fixed_int(u, e);
  if (a != b) return 0;
  int32_t d[lg::kSlices];
  lg::slice_digits(a, d);
  const uint64_t Y = lg::slice_bias(b);
  for (int i = 0; i < lg::kSlices; ++i)
    if (lg::slice_digit(b, Y, i) != d[i]) return 0;
  return 1;
}

// levels_to_double on (hi, lo, E): returns 1 and the double, or 0 when the
// integer route declines (subnormal / overflow)
int h_levels_to_double(int64_t hi, int64_t lo, int E, double* out) { return lg::levels_to_double(hi, lo, E, out) ? 1 : 0; }

// the 32-bit conversion against the 128-bit one on the same levels: 1 if both
// give the same result (or both refuse)
int h_levels32_agree(const int32_t* c, int E) {
  int64_t hi, lo;
  lg::level_halves(c, &hi, &lo);
  double a = 0.0, b = 0.0;
  const bool ra = lg::levels_to_double(hi, lo, E, &a), rb = lg::levels_to_double32(c, E, &b);
  if (ra != rb) return 0;
  return (!ra || a == b) ? 1 : 0;
}

// the two epilogue routes on the same levels: FP64 (combine_levels_add) and integer
void h_combine_both(const int32_t* c, int32_t eu, int32_t ev, double w, double* out2) {
  out2[0] = lg::combine_levels_add(c, eu, ev, w);
  out2[1] = lg::combine_levels_add_int(c, eu, ev, w);
  if (lg::combine_levels_int32(c, eu, ev) != lg::combine_levels_int(c, eu, ev)) out2[1] = -out2[1] - 1.0;
  if (lg::combine_levels_fp(c, eu, ev) != lg::combine_levels_int(c, eu, ev)) out2[1] = -out2[1] - 2.0;
}
double h_small_int_to_double(int64_t x) { return lg::small_int_to_double(x); }
int32_t h_slice_exponent(double m) { return lg::slice_exponent(m); }
}
