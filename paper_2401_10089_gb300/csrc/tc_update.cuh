// tc_update.cuh -- the rank-32 Gauss-Jordan update of the whole-GPU kernel,
// W[:, not J] += (P_f - I_J) R, on the tensor cores with FP64 accuracy.
//
// The panel's two factors are split into exact BF16 digits (fp64_slices.cuh):
// U = P_f - I_J row by row, V = R column by column, eight digits each, stored
// K-major in global memory (kDigK = 8 x 32 BF16 per row or column). Each
// block then runs its share of the 128 x 64 output tiles of W:
//   * TMA copies the tile's U digits (128 x 256 BF16, four 128-byte swizzle
//     boxes) and V digits (64 x 256) into shared memory; the V copy of the next
//     tile overlaps the current tile's epilogue (two stages);
//   * one thread issues 72 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//     M = 128, N = 64, K = 16): for every level L = i + j of the digit pairs
//     (i, j), both K halves of the 32 terms, accumulated into its own TMEM
//     region of 64 columns (8 levels = all 512 columns). Every level sum is an
//     integer below 2^22, so the FP32 accumulation is exact;
//   * all eight warps read the levels back (tcgen05.ld), combine them into the
//     exact integer dot product, round it to FP64 once and add it to W.
// Per element and panel that is 4 FP64 instructions instead of 32 FP64 FMAs.
//
// Every mbarrier wait is bounded (kTmWaitLimit polls); a wait that runs out
// sets the grid's error word, and the kernel reports LOGM_INFO_TIMEOUT for the
// matrix instead of hanging.
#pragma once

#include <cuda_bf16.h>

#include "fp64_slices.cuh"
#include "tc_ptx.cuh"

namespace lg {

constexpr int kUpdM = 128, kUpdN = 64;                      // output tile of W: rows x columns
constexpr int kDigK = kSlices * kSliceK;                    // digits per row of U / column of V
constexpr uint32_t kUpdABytes = kUpdM * kDigK * 2;          // 64 KB
constexpr uint32_t kUpdBBytes = kUpdN * kDigK * 2;          // 32 KB
constexpr uint32_t kUpdAtomA = kUpdM * 128, kUpdAtomB = kUpdN * 128;  // one 128-byte swizzle box
constexpr size_t kUpdSmemBytes = kUpdABytes + 2 * kUpdBBytes + 1024;  // + alignment slack
constexpr int kUpdTmemCols = kSliceLevels * kUpdN;           // 512
static_assert(kUpdTmemCols == 512, "eight levels of 64 columns fill TMEM");

// Tensor maps of the digit buffers, per inversion group (2-D: kDigK x n_max
// BF16, boxes of 64 x 128 rows for U and 64 x 64 for V, 128-byte swizzle).
struct SliceMaps {
  CUtensorMap a[2];
  CUtensorMap b[2];
};

struct SliceBufs {
  __nv_bfloat16* adig;  // [n_max][kDigK]: row r of U, digit i of term k at [r][32 i + k]
  __nv_bfloat16* bdig;  // [n_max][kDigK]: column j of V likewise
  int32_t* aexp;        // [n_max] scale exponent of each row of U
  int32_t* bexp;        // [n_max] scale exponent of each column of V
};

struct SliceSmem {
  unsigned long long bar[4];  // U tile full, V stage 0 full, V stage 1 full, accumulators ready
  uint32_t phase[4];          // completed phases of each barrier
  uint32_t tmem;              // TMEM base address of the level accumulators
  int failed;                 // a bounded wait ran out
};

// The digits of 32 values (the first `count` given, the rest zero), stored
// as one row of kDigK BF16 at out; the scale exponent goes to *eo.
static __device__ void slice_store(const double* v, int count, __nv_bfloat16* out, int32_t* eo) {
  double m = 0.0;
  for (int k = 0; k < count; ++k) {
    const double a = fabs(v[k]);
    if (!(a <= m)) m = a;  // NaN wins
  }
  const int32_t e = slice_exponent(m);
  *eo = e;
  int64_t X[kSliceK];
  for (int k = 0; k < kSliceK; ++k) X[k] = (k < count && e != kSliceNonFinite) ? slice_fixed(v[k], e) : 0;
  uint4* o = reinterpret_cast<uint4*>(out);
  // least significant digit first; digit i of every term fills 32 BF16 (4 x 16 B)
  for (int i = kSlices - 1; i >= 0; --i) {
    uint32_t pk[kSliceK / 2];
    for (int k = 0; k < kSliceK; k += 2) {
      int32_t d0, d1;
      if (i > 0) {
        d0 = static_cast<int32_t>((X[k] + 128) & 255) - 128;
        d1 = static_cast<int32_t>((X[k + 1] + 128) & 255) - 128;
        X[k] = (X[k] - d0) / 256;
        X[k + 1] = (X[k + 1] - d1) / 256;
      } else {
        d0 = static_cast<int32_t>(X[k]);
        d1 = static_cast<int32_t>(X[k + 1]);
      }
      // |d| <= 128 has at most 8 significant bits: the BF16 is the FP32's top half
      pk[k / 2] = (__float_as_uint(static_cast<float>(d0)) >> 16) |
                  (__float_as_uint(static_cast<float>(d1)) & 0xFFFF0000u);
    }
    for (int q = 0; q < 4; ++q) o[i * 4 + q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
  }
}

// Generic-proxy writes (the digits) made visible to later TMA reads.
static __device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// W[r, c] += (U V)[r, c] for every r < n and every column c < n outside
// [kb, kb + jb), over the tiles [t_lo, t_hi) of this block (row-major order
// of the ceil(n / 128) x ceil(n / 64) tiles). dyn: this block's dynamic shared
// memory; err: the grid's error word.
static __device__ void sliced_update(SliceSmem& sm, unsigned char* dyn, const CUtensorMap* map_a,
                                     const CUtensorMap* map_b, const SliceBufs& sb, double* W, int n, int kb, int jb,
                                     int t_lo, int t_hi, int* err) {
  if (t_lo >= t_hi) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncb = (n + kUpdN - 1) / kUpdN;
  const uint32_t raw = su32(dyn);
  const uint32_t sA = (raw + 1023u) & ~1023u;
  const uint32_t sB[2] = {sA + kUpdABytes, sA + kUpdABytes + kUpdBBytes};
  const uint32_t barA = su32(&sm.bar[0]), barB[2] = {su32(&sm.bar[1]), su32(&sm.bar[2])}, barAcc = su32(&sm.bar[3]);
  uint32_t phA = sm.phase[0], phB[2] = {sm.phase[1], sm.phase[2]}, phAcc = sm.phase[3];
  const uint32_t tmem = sm.tmem;
  __syncthreads();  // everyone has read the phases

  auto issue = [&](int t, bool with_a, int st) {
    const int rb = t / ncb, cb = t % ncb;
    if (with_a) {
      tm_expect(barA, kUpdABytes);
      for (int a = 0; a < 4; ++a) tm_load2d(sA + a * kUpdAtomA, map_a, barA, a * 64, rb * kUpdM);
    }
    tm_expect(barB[st], kUpdBBytes);
    for (int a = 0; a < 4; ++a) tm_load2d(sB[st] + a * kUpdAtomB, map_b, barB[st], a * 64, cb * kUpdN);
  };

  // thread 0: phases issued on each barrier (lifetime counts, like phA ...)
  uint32_t isA = phA, isB[2] = {phB[0], phB[1]}, isAcc = phAcc;
  if (tid == 0) {
    issue(t_lo, true, 0);
    ++isA;
    ++isB[0];
  }
  bool failed = false;
  for (int t = t_lo; t < t_hi; ++t) {
    const int k = t - t_lo, st = k & 1;
    const int rb = t / ncb, cb = t % ncb;
    const bool new_a = (t == t_lo) || (rb != (t - 1) / ncb);
    const bool has_next = t + 1 < t_hi;
    const bool next_new_a = has_next && ((t + 1) / ncb != rb);
    if (tid == 32) {  // the MMA issuer
      bool ok = true;
      if (new_a) ok = tm_wait(barA, phA & 1);
      ok = ok && tm_wait(barB[st], phB[st] & 1);
      if (ok) {
        tm_fence_after();
        const uint32_t id = tm_idesc(1, kUpdM, kUpdN);  // BF16 x BF16 -> FP32
        for (int L = 2; L <= kSlices + 1; ++L) {
          int first = 1;
          for (int i = 1; i < L; ++i) {
            const int j = L - i;
            for (int h = 0; h < 2; ++h) {
              const int ka = 32 * (i - 1) + 16 * h, kbb = 32 * (j - 1) + 16 * h;
              const uint64_t da = tm_desc(sA + (ka / 64) * kUpdAtomA + (ka % 64) * 2);
              const uint64_t db = tm_desc(sB[st] + (kbb / 64) * kUpdAtomB + (kbb % 64) * 2);
              tm_mma_f16(tmem + static_cast<uint32_t>((L - 2) * kUpdN), da, db, id, first ? 0 : 1);
              first = 0;
            }
          }
        }
      } else {
        atomicExch(&sm.failed, 1);
      }
      tm_commit(barAcc);  // arrives once the MMAs issued so far are complete
    }
    if (new_a) ++phA;
    ++phB[st];
    ++isAcc;  // one commit per tile
    if (tid == 0 && has_next && !next_new_a) {  // the other V stage is free: its last reader was tile t - 1
      issue(t + 1, false, st ^ 1);
      ++isB[st ^ 1];
    }
    // tcgen05.ld is warp-collective: a warp reads the accumulators only if all its lanes saw them ready
    const bool acc_ok = __all_sync(0xffffffffu, tm_wait(barAcc, phAcc & 1));
    ++phAcc;
    tm_fence_after();
    if (!acc_ok) atomicExch(&sm.failed, 1);
    if (tid == 0 && has_next && next_new_a) {  // the U tile is free once this tile's MMAs are done
      issue(t + 1, true, st ^ 1);
      ++isA;
      ++isB[st ^ 1];
    }
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows), columns half (w / 4)
    const int lbase = (warp & 3) * 32, half = warp >> 2;
    const int row = rb * kUpdM + lbase + lane;
    const int c0 = cb * kUpdN;
    const int32_t er = row < n ? sb.aexp[row] : 0;
    double* Wrow = W + (int64_t)row * n;
    if (acc_ok) {
      for (int q = 0; q < 4; ++q) {
        const int cc = half * 32 + q * 8;
        uint32_t v[kSliceLevels][8];
        for (int L = 0; L < kSliceLevels; ++L)
          tm_ld8(tmem + (static_cast<uint32_t>(lbase) << 16) + static_cast<uint32_t>(L * kUpdN + cc), v[L]);
        tm_ld_wait();
        if (row < n) {
          for (int e = 0; e < 8; ++e) {
            const int gc = c0 + cc + e;
            if (gc >= n || (gc >= kb && gc < kb + jb)) continue;
            int32_t c[kSliceLevels];
            for (int L = 0; L < kSliceLevels; ++L) c[L] = level_int(__uint_as_float(v[L][e]));
            Wrow[gc] = combine_levels_add(c, er, sb.bexp[gc], Wrow[gc]);
          }
        }
      }
    }
    tm_fence_before();
    __syncthreads();
    failed = sm.failed != 0;
    if (failed) break;
  }
  if (failed) {
    // wait (bounded) for this block's copies and MMAs still in flight: the
    // last phase issued on each barrier (a completed phase returns at once)
    if (tid == 0) {
      if (isA > sm.phase[0]) tm_wait(barA, (isA - 1) & 1);
      for (int s = 0; s < 2; ++s)
        if (isB[s] > sm.phase[1 + s]) tm_wait(barB[s], (isB[s] - 1) & 1);
      if (isAcc > sm.phase[3]) tm_wait(barAcc, (isAcc - 1) & 1);
      atomicExch(err, 1);
    }
  }
  if (tid == 0) {
    // the phases this block's barriers have completed (after a failure they
    // no longer matter: the kernel skips every later update)
    sm.phase[0] = phA;
    sm.phase[1] = phB[0];
    sm.phase[2] = phB[1];
    sm.phase[3] = phAcc;
  }
  __syncthreads();
}

}  // namespace lg
