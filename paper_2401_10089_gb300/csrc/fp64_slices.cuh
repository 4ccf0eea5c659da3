// fp64_slices.cuh -- FP64 products from exact BF16 digit products.
//
// A product C = U V of FP64 matrices (K <= kSliceK terms per entry) is formed
// from small integers so that the BF16 tensor cores compute it exactly:
//
//  * every row u of U (every column v of V) is scaled by its own power of two
//    2^-e, e the smallest integer with max_k |u_k| < 2^e, and rounded to a
//    fixed-point integer X_k = round(u_k 2^(F - e)), F = 7 + 8 (kSlices - 1);
//  * X_k is written in balanced base 256 with kSlices digits,
//    X_k = sum_i d_i 256^(kSlices - i), d_1 in [-128, 128], the others in
//    [-128, 127]: each digit is exact in BF16 (8 significant bits);
//  * digit products d_i e_j are at most 2^14 in magnitude, so for a level
//    L = i + j the sum over the pairs of that level and over K = 32 terms,
//    C_L = sum_{i + j = L} sum_k d_i[k] e_j[k], is an integer of magnitude
//    <= 8 * 32 * 2^14 = 2^22: FP32 accumulation on the tensor cores is exact;
//  * u.v = 2^(e_u + e_v - 14 - 8 (kSlices - 1)) * T with the integer
//    T = sum_{L = 2}^{kSlices + 1} C_L 256^(kSlices + 1 - L) (pairs with
//    i + j > kSlices + 1 weigh less than 2^-76 of the row/column scale and are
//    dropped). T is combined from the FP32 levels with integer arithmetic and
//    converted to FP64 with two roundings.
//
// The split error is at most 2^-(F+1) of the row or column scale per operand
// (2^-64 for kSlices = 8), below FP64's own rounding of the result. The
// helpers are __host__ __device__ so that the CPU tests exercise the same code.
#pragma once

#include <cstdint>
#include <cmath>
#include <cstring>

#ifdef __CUDACC__
#define LG_HD __host__ __device__ __forceinline__
#else
#define LG_HD inline
#endif

namespace lg {

constexpr int kSlices = 8;                     // digits per operand (slice_bias assumes 8)
constexpr int kSliceK = 32;                    // K of one exact accumulation (the panel width)
constexpr int kSliceLevels = kSlices;          // levels L = 2 .. kSlices + 1
constexpr int kSliceFrac = 7 + 8 * (kSlices - 1);  // F: fractional bits of the fixed-point form
constexpr int kSliceScale = 14 + 8 * (kSlices - 1);  // u.v = 2^(e_u + e_v - kSliceScale) T
constexpr int32_t kSliceNonFinite = -0x40000000;   // exponent marker of a row/column with Inf or NaN

LG_HD uint64_t lg_dbits(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
}
LG_HD double lg_bitsd(uint64_t b) {
  double x;
  memcpy(&x, &b, 8);
  return x;
}
LG_HD uint32_t lg_fbits(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  return b;
}

// 2^e as a double for e in [-1022, 1023] (exact).
LG_HD double lg_pow2(int e) { return lg_bitsd(static_cast<uint64_t>(e + 1023) << 52); }

// Scale exponent of a row or column: the smallest e with max|u_k| < 2^e for
// the finite maximum m > 0; 0 when m == 0; kSliceNonFinite for Inf or NaN.
LG_HD int32_t slice_exponent(double m) {
  if (!(m <= 1.79769313486231570815e308)) return kSliceNonFinite;  // Inf or NaN
  if (m == 0.0) return 0;
  const uint64_t b = lg_dbits(m);
  const int be = static_cast<int>((b >> 52) & 0x7FF);
  if (be != 0) return be - 1023 + 1;  // m in [2^(be-1023), 2^(be-1022))
  // subnormal: m = frac * 2^-1074, frac < 2^52
  const uint64_t frac = b & ((1ull << 52) - 1);
  int top = 63;
  while (!((frac >> top) & 1ull)) --top;
  return -1074 + top + 1;
}

// Fixed-point integer round(u 2^(kSliceFrac - e)), |result| < 2^63 for |u| < 2^e.
LG_HD int64_t slice_fixed(double u, int32_t e) {
  // u 2^(F - e) computed as (u 2^-e) 2^F: exact scalings by powers of two, in
  // two steps so that neither factor over- or underflows for e in the double range
  const int sh = kSliceFrac - e;  // may be up to about 63 + 1074
  double y = u;
  int rest = sh;
  while (rest > 1000) {
    y *= lg_pow2(1000);
    rest -= 1000;
  }
  while (rest < -1000) {
    y *= lg_pow2(-1000);
    rest += 1000;
  }
  y *= lg_pow2(rest);
#ifdef __CUDA_ARCH__
  return __double2ll_rn(y);
#else
  return static_cast<int64_t>(std::nearbyint(y));
#endif
}

// Balanced base-256 digits of X, most significant first: d[0] in [-128, 128],
// d[1..] in [-128, 127], X = sum d[i] 256^(kSlices - 1 - i).
LG_HD void slice_digits(int64_t X, int32_t* d) {
  for (int i = kSlices - 1; i >= 1; --i) {
    const int32_t di = static_cast<int32_t>((X + 128) & 255) - 128;
    d[i] = di;
    X = (X - di) / 256;  // exact: X - di is a multiple of 256
  }
  d[0] = static_cast<int32_t>(X);
}

// The same integer as slice_fixed (round(u 2^(kSliceFrac - e)), ties to
// even) from the bits of u with integer operations only: u = M 2^(x - 52)
// with the 53-bit integer M, so the result is M shifted by x - 52 + F - e
// (at most 10 to the left, since |u| < 2^e), rounded when shifted right.
LG_HD int64_t slice_fixed_int(double u, int32_t e) {
  const uint64_t b = lg_dbits(u);
  const int bx = static_cast<int>((b >> 52) & 0x7FF);
  uint64_t M = b & ((1ull << 52) - 1);
  int x;
  if (bx == 0) {
    x = -1022;  // subnormal (or zero): no implicit bit
  } else {
    M |= 1ull << 52;
    x = bx - 1023;
  }
  const int sh = x - 52 + kSliceFrac - e;
  uint64_t mag;
  if (sh >= 0) {
    mag = M << sh;  // sh <= 10: below 2^63
  } else if (sh > -64) {
    const int r = -sh;
    const uint64_t q = M >> r, rem = M & ((1ull << r) - 1), half = 1ull << (r - 1);
    mag = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
  } else {
    mag = 0;  // below half a unit of the last digit
  }
  return (b >> 63) ? -static_cast<int64_t>(mag) : static_cast<int64_t>(mag);
}

// Digit i (0 = most significant) of the balanced base-256 form of X (the
// digits slice_digits gives), without the carry chain: with the bias
// C = sum of 128 * 256^m (m = 0 .. kSlices - 2), digit m from the bottom is
// byte m of X + C minus 128, and the top digit is (X + C) >> 8 (kSlices - 1).
// Y = X + C is kept modulo 2^64 (|X| may reach 2^63 - 2^10); the top digit
// is formed from X itself and the carry of its low bytes.
constexpr uint64_t kSliceBias = 0x0080808080808080ull;
LG_HD uint64_t slice_bias(int64_t X) { return static_cast<uint64_t>(X) + kSliceBias; }
LG_HD int32_t slice_digit(int64_t X, uint64_t Y, int i) {
  constexpr int top = 8 * (kSlices - 1);
  if (i == 0) {
    const uint64_t low = static_cast<uint64_t>(X) & ((1ull << top) - 1);
    return static_cast<int32_t>(X >> top) + static_cast<int32_t>((low + kSliceBias) >> top);
  }
  return static_cast<int32_t>((Y >> (8 * (kSlices - 1 - i))) & 255) - 128;
}

// Integer value of an FP32 level sum (an exact integer, |v| <= 2^22).
LG_HD int32_t level_int(float v) {
  return static_cast<int32_t>(lg_fbits(v + 12582912.0f)) - 0x4B400000;
}

// Integer value of an FP32 level sum accumulated over up to four chunks of
// 32 terms (an exact integer, |v| <= 2^24): split as v = h 2^12 + l with
// |h| <= 2^12 and |l| <= 2^11, each converted by the magic-number addition.
LG_HD int32_t level_int_wide(float v) {
  const float hf = (v * 2.44140625e-4f + 12582912.0f) - 12582912.0f;  // rint(v 2^-12), exact
  const float lf = fmaf(-hf, 4096.0f, v);                              // exact remainder
  return level_int(hf) * 4096 + level_int(lf);
}

// Exact integer T = sum_L C_L 256^(kSlices + 1 - L) as two halves,
// T = hi 2^32 + lo, from the kSlices level sums c[0] (L = 2) .. c[kSlices-1].
LG_HD void level_halves(const int32_t* c, int64_t* hi, int64_t* lo) {
  static_assert(kSlices == 8, "two halves of four levels each");
  *hi = ((static_cast<int64_t>(c[0]) * 256 + c[1]) * 256 + c[2]) * 256 + c[3];
  *lo = ((static_cast<int64_t>(c[4]) * 256 + c[5]) * 256 + c[6]) * 256 + c[7];
}

// Exact FP64 value of an integer with |x| < 2^51.
LG_HD double small_int_to_double(int64_t x) {
  return lg_bitsd(static_cast<uint64_t>(x + 0x4338000000000000ll)) - 6755399441055744.0;
}

// u.v from the levels and the two scale exponents (both finite markers):
// T rounded to FP64 once, then scaled exactly (unless it under- or overflows).
LG_HD double combine_levels(const int32_t* c, int32_t eu, int32_t ev) {
  if (eu == kSliceNonFinite || ev == kSliceNonFinite) return lg_bitsd(0x7FF8000000000000ull);  // NaN
  int64_t hi, lo;
  level_halves(c, &hi, &lo);
  const double t = fma(small_int_to_double(hi), 4294967296.0, small_int_to_double(lo));
  const int E = eu + ev - kSliceScale;
  if (E >= -1022 && E <= 1023) return t * lg_pow2(E);
  return ldexp(t, E);  // rare: the scale itself is outside the normal range
}

// Leading zeros of a 64-bit word (x != 0).
LG_HD int lg_clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(x));
#else
  return __builtin_clzll(x);
#endif
}

// (hi 2^32 + lo) 2^E rounded to the nearest FP64 (ties to even) with integer
// operations only (no FP64 instruction): the signed 128-bit sum, its
// magnitude normalised, 53 bits kept with round/sticky bits, the exponent
// field set to the binary point plus E. hi, lo as from level_halves
// (|hi|, |lo| < 2^48). Returns false (leaving *out alone) when the result
// would be subnormal or overflow; the caller then takes the FP64 route.
LG_HD bool levels_to_double(int64_t hi, int64_t lo, int E, double* out) {
  // 128-bit two's complement value v = hi 2^32 + lo as (vh, vl)
  const uint64_t a_lo = static_cast<uint64_t>(hi) << 32;
  const uint64_t a_hi = static_cast<uint64_t>(hi >> 32);  // arithmetic shift: sign extension
  const uint64_t b_lo = static_cast<uint64_t>(lo);
  const uint64_t b_hi = static_cast<uint64_t>(lo >> 63);
  uint64_t vl = a_lo + b_lo;
  uint64_t vh = a_hi + b_hi + (vl < a_lo ? 1u : 0u);
  const uint64_t sign = vh >> 63;
  if (sign) {  // magnitude
    vl = ~vl + 1;
    vh = ~vh + (vl == 0 ? 1u : 0u);
  }
  if ((vh | vl) == 0) {
    *out = 0.0;
    return true;
  }
  // normalise: the leading one to bit 127
  int lz;
  if (vh != 0) {
    lz = lg_clz64(vh);
    if (lz) {
      vh = (vh << lz) | (vl >> (64 - lz));
      vl <<= lz;
    }
  } else {
    lz = 64 + lg_clz64(vl);
    vh = vl << (lz - 64);
    vl = 0;
  }
  // 53 bits of mantissa, then the guard bit and the sticky bits
  uint64_t m = vh >> 11;
  const uint64_t guard = (vh >> 10) & 1u;
  const bool sticky = ((vh & 0x3FFu) | vl) != 0;
  int p = 127 - lz;  // position of the leading one in the integer
  if (guard && (sticky || (m & 1u))) {
    m += 1;
    if (m >> 53) {
      m >>= 1;
      ++p;
    }
  }
  const int be = p + E + 1023;  // biased exponent of m 2^(p - 52) 2^E
  if (be < 1 || be > 2046) return false;
  *out = lg_bitsd((sign << 63) | (static_cast<uint64_t>(be) << 52) | (m & ((1ull << 52) - 1)));
  return true;
}

// w + u.v with the same two roundings (T to FP64, then the sum: one FMA).
LG_HD double combine_levels_add(const int32_t* c, int32_t eu, int32_t ev, double w) {
  if (eu == kSliceNonFinite || ev == kSliceNonFinite) return lg_bitsd(0x7FF8000000000000ull);  // NaN
  int64_t hi, lo;
  level_halves(c, &hi, &lo);
  const double t = fma(small_int_to_double(hi), 4294967296.0, small_int_to_double(lo));
  const int E = eu + ev - kSliceScale;
  if (E >= -1022 && E <= 1023) return fma(t, lg_pow2(E), w);
  return w + ldexp(t, E);
}

// 32-bit helpers (funnel shift left of (hi:lo) by 0..31; leading zeros)
LG_HD uint32_t lg_shl64hi(uint32_t hi, uint32_t lo, int s) {
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lo, hi, s);
#else
  return s == 0 ? hi : (hi << s) | (lo >> (32 - s));
#endif
}
LG_HD int lg_clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz(static_cast<int>(x));
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// T 2^E rounded to the nearest FP64 (ties to even) with 32-bit integer
// operations only and no branches on data, T = sum_L c[L - 2] 256^(9 - L)
// from the eight level sums (|c| <= 2^22). The same result as
// levels_to_double(level_halves(c), E), the same refusal (false) for a
// subnormal or overflowing result.
//   The levels pair into four 31-bit words P1 = c0 256 + c1 .. P4 = c6 256 + c7
// with T = P1 2^48 + P2 2^32 + P3 2^16 + P4, summed into a 96-bit two's
// complement (w2:w1:w0) with carries; then magnitude, normalisation by
// funnel shifts, round to nearest even, and the IEEE bit pattern assembled
// so that a rounding carry moves into the exponent field by itself.
LG_HD bool levels_to_double32(const int32_t* c, int E, double* out) {
  static_assert(kSlices == 8, "eight levels");
  const int32_t P1 = c[0] * 256 + c[1], P2 = c[2] * 256 + c[3];
  const int32_t P3 = c[4] * 256 + c[5], P4 = c[6] * 256 + c[7];
  // 96-bit sum of P4, P3 << 16, P2 << 32, P1 << 48, each sign-extended
  const uint32_t s4 = static_cast<uint32_t>(P4 >> 31), s3 = static_cast<uint32_t>(P3 >> 31);
  const uint32_t s2 = static_cast<uint32_t>(P2 >> 31), s1 = static_cast<uint32_t>(P1 >> 31);
  // word 0: P4 + (P3 << 16)
  const uint32_t a0 = static_cast<uint32_t>(P4), b0 = static_cast<uint32_t>(P3) << 16;
  uint32_t w0 = a0 + b0;
  uint32_t cy = w0 < a0;
  // word 1: s4 + (P3 >> 16) + P2 + (P1 << 16) + carry
  const uint32_t b1 = static_cast<uint32_t>(P3 >> 16), c1 = static_cast<uint32_t>(P2),
                 d1 = static_cast<uint32_t>(P1) << 16;
  uint64_t t1 = static_cast<uint64_t>(s4) + b1 + c1 + d1 + cy;
  uint32_t w1 = static_cast<uint32_t>(t1);
  // word 2: s4 + s3 + s2 + (P1 >> 16) + carries of word 1
  uint32_t w2 = s4 + s3 + s2 + static_cast<uint32_t>(P1 >> 16) + static_cast<uint32_t>(t1 >> 32);
  (void)s1;
  // magnitude
  const uint32_t neg = static_cast<uint32_t>(static_cast<int32_t>(w2) >> 31);  // all ones if negative
  w0 ^= neg;
  w1 ^= neg;
  w2 ^= neg;
  const uint64_t u0 = static_cast<uint64_t>(w0) + (neg & 1u);
  w0 = static_cast<uint32_t>(u0);
  const uint64_t u1 = static_cast<uint64_t>(w1) + static_cast<uint32_t>(u0 >> 32);
  w1 = static_cast<uint32_t>(u1);
  w2 += static_cast<uint32_t>(u1 >> 32);
  // normalise: the leading one to bit 95 of (x2:x1:x0)
  const bool top0 = w2 == 0;
  uint32_t x2 = top0 ? w1 : w2, x1 = top0 ? w0 : w1, x0 = top0 ? 0u : w0;
  int lz = lg_clz32(x2);
  const bool top1 = top0 && x2 == 0;  // w2 = w1 = 0: move one more word
  if (top1) {
    x2 = x1;
    x1 = 0;
    x0 = 0;
    lz = lg_clz32(x2);
  }
  if (x2 == 0) {  // T = 0
    *out = 0.0;
    return true;
  }
  const int sh = lz & 31;
  const uint32_t y2 = lg_shl64hi(x2, x1, sh), y1 = lg_shl64hi(x1, x0, sh), y0 = x0 << sh;
  const int p = 95 - lz - (top0 ? 32 : 0) - (top1 ? 32 : 0);  // position of the leading one in T
  // 53 bits: y2 (32) and the top 21 of y1; guard = bit 10 of y1; sticky = the rest
  const uint32_t guard = (y1 >> 10) & 1u;
  const uint32_t sticky = ((y1 & 0x3FFu) | y0) != 0u;
  const uint32_t mlo = (y1 >> 11) | (y2 << 21);  // mantissa bits 0..31
  const uint32_t mhi = y2 >> 11;                  // mantissa bits 32..52 (bit 20 = the leading one)
  const int be = p + E + 1023;
  if (be < 1 || be > 2046) return false;
  // bit pattern without the implicit one, then the rounding increment (its
  // carry may reach the exponent: that is the correct rounding up)
  const uint32_t inc = guard & (sticky | (mlo & 1u));
  const uint64_t bits = ((static_cast<uint64_t>(neg & 1u) << 63) | (static_cast<uint64_t>(be) << 52) |
                         (static_cast<uint64_t>(mhi & 0xFFFFFu) << 32) | mlo) +
                        inc;
  if (((bits >> 52) & 0x7FF) == 0x7FF) return false;  // rounded up to Inf
  *out = lg_bitsd(bits);
  return true;
}

// u.v with T rounded to FP64 by integer operations (no FP64 instruction
// unless the product is subnormal or overflows).
LG_HD double combine_levels_int(const int32_t* c, int32_t eu, int32_t ev) {
  if (eu == kSliceNonFinite || ev == kSliceNonFinite) return lg_bitsd(0x7FF8000000000000ull);  // NaN
  int64_t hi, lo;
  level_halves(c, &hi, &lo);
  double t;
  if (levels_to_double(hi, lo, eu + ev - kSliceScale, &t)) return t;
  return combine_levels(c, eu, ev);
}

// Exact FP64 value of an integer with |x| < 2^53, built with integer
// operations (sign, leading zeros, shift, exponent field): no FP64 instruction.
LG_HD double exact_int_to_double(int64_t x) {
  const uint64_t sgn = static_cast<uint64_t>(x >> 63);
  const uint64_t a = (static_cast<uint64_t>(x) ^ sgn) - sgn;  // |x|
  if (a == 0) return 0.0;
  const int lz = lg_clz64(a);                                  // >= 11
  const uint64_t m = a << (lz - 11);                           // leading one at bit 52
  const uint64_t be = static_cast<uint64_t>(1023 + 63 - lz);
  return lg_bitsd((sgn << 63) | (be << 52) | (m & ((1ull << 52) - 1)));
}

// Exact FP64 value of an integer with |x| < 2^51: the hardware conversion on
// the device (measured a little faster than the magic-number addition on
// GB300), the magic-number addition on the host.
LG_HD double half_to_double(int64_t x) {
#ifdef __CUDA_ARCH__
  return __ll2double_rn(x);
#else
  return small_int_to_double(x);
#endif
}

// u.v as combine_levels_int through the FP64 pipe: the two halves of T
// (below 2^50 in magnitude for level sums up to 2^24) converted exactly and
// joined by one FMA (one rounding, the same result), the scale 2^E added to
// the exponent field with an integer addition. On GB300 this measured faster
// than the all-integer routes (whose 64-bit variable shifts cost more issue
// slots than the FP64 pipe time they save).
LG_HD double combine_levels_fp(const int32_t* c, int32_t eu, int32_t ev) {
  if (eu == kSliceNonFinite || ev == kSliceNonFinite) return lg_bitsd(0x7FF8000000000000ull);  // NaN
  int64_t hi, lo;
  level_halves(c, &hi, &lo);
  if ((hi | lo) == 0) return 0.0;
  const double t = fma(half_to_double(hi), 4294967296.0, half_to_double(lo));
  const int E = eu + ev - kSliceScale;
  const uint64_t b = lg_dbits(t);
  const int be = static_cast<int>((b >> 52) & 0x7FF) + E;
  if (be >= 1 && be <= 2046) return lg_bitsd(b + (static_cast<uint64_t>(static_cast<int64_t>(E)) << 52));
  return ldexp(t, E);  // rare: subnormal or overflowing result
}

// combine_levels_fp without branches for the common case: *slow is set
// when the result needs combine_levels_fp instead (a non-finite row or
// column, or a subnormal or overflowing result); the value returned is then
// meaningless.
LG_HD double combine_levels_fast(const int32_t* c, int32_t eu, int32_t ev, bool* slow) {
  int64_t hi, lo;
  level_halves(c, &hi, &lo);
  const double t = fma(half_to_double(hi), 4294967296.0, half_to_double(lo));
  const int E = eu + ev - kSliceScale;
  const uint64_t b = lg_dbits(t);
  const int be = static_cast<int>((b >> 52) & 0x7FF) + E;
  const bool zero = (hi | lo) == 0;
  *slow = (!zero && (be < 1 || be > 2046)) || eu == kSliceNonFinite || ev == kSliceNonFinite;
  return zero ? 0.0 : lg_bitsd(b + (static_cast<uint64_t>(static_cast<int64_t>(E)) << 52));
}

// u.v as combine_levels_int, with the branch-free 32-bit conversion.
LG_HD double combine_levels_int32(const int32_t* c, int32_t eu, int32_t ev) {
  if (eu == kSliceNonFinite || ev == kSliceNonFinite) return lg_bitsd(0x7FF8000000000000ull);  // NaN
  double t;
  if (levels_to_double32(c, eu + ev - kSliceScale, &t)) return t;
  return combine_levels(c, eu, ev);
}

// w + u.v with T rounded to FP64 by integer operations (one FP64 instruction
// per element: the addition), the same two roundings as combine_levels_add.
LG_HD double combine_levels_add_int(const int32_t* c, int32_t eu, int32_t ev, double w) {
  if (eu == kSliceNonFinite || ev == kSliceNonFinite) return lg_bitsd(0x7FF8000000000000ull);  // NaN
  int64_t hi, lo;
  level_halves(c, &hi, &lo);
  double t;
  if (levels_to_double(hi, lo, eu + ev - kSliceScale, &t)) return w + t;
  return combine_levels_add(c, eu, ev, w);  // subnormal or overflowing product: the FP64 route
}

}  // namespace lg
