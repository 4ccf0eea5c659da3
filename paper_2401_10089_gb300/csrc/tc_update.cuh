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
//     exact integer dot product and round it to FP64 (integer operations and
//     three FP64 instructions) into a shared-memory tile; the next tile's MMAs start as soon as TMEM is
//     read, while the warps add the staged tile to W row by row (coalesced).
// Per element and panel that is four FP64 instructions (the conversion and
// the addition) instead of 32 FP64 FMAs.
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
constexpr int kUpdTsStride = kUpdN + 1;                     // staged tile: doubles per row (padded)
constexpr uint32_t kUpdTsBytes = kUpdM * kUpdTsStride * 8;   // 65 KB
constexpr size_t kUpdSmemBytes = kUpdABytes + 2 * kUpdBBytes + kUpdTsBytes + 1024;  // + alignment slack
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
  int32_t ecol[kUpdN];        // scale exponents of the current tile's columns of V
};

// The digits of one row of 32 values split among the 8 lanes of an aligned
// lane group (lanes 8q .. 8q + 7 of a warp): lane i holds the values
// k = 4 i .. 4 i + 3 (zero past the row's length) in v0..v3. The group forms the
// row's scale exponent (the largest magnitude by integer comparison of the
// bit patterns: NaN above Inf above every finite value), each lane the
// fixed-point integers and all eight digits of its four values, and writes
// them as eight 8-byte pieces of the row of kDigK BF16 at out (digit s of
// value k at out[32 s + k]); lane 0 stores the exponent at *eo. Every lane
// of the warp must call this (the shuffles); `valid` lanes store.
static __device__ __noinline__ void slice_row8(double v0, double v1, double v2, double v3, int i, bool valid,
                                               __nv_bfloat16* out, int32_t* eo) {
  const double v[4] = {v0, v1, v2, v3};
  unsigned long long mb = 0;
  for (int t = 0; t < 4; ++t) {
    const unsigned long long a = lg_dbits(v[t]) & 0x7FFFFFFFFFFFFFFFull;
    mb = a > mb ? a : mb;
  }
  for (int x = 1; x < 8; x <<= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, mb, x);
    mb = o > mb ? o : mb;
  }
  const int32_t e = slice_exponent(lg_bitsd(mb));
  if (valid && i == 0) *eo = e;
  int64_t X[4];
  uint64_t Y[4];
  for (int t = 0; t < 4; ++t) {
    X[t] = e != kSliceNonFinite ? slice_fixed_int(v[t], e) : 0;
    Y[t] = slice_bias(X[t]);
  }
  if (!valid) return;
  for (int sl = 0; sl < kSlices; ++sl) {
    uint32_t b[4];
    // |d| <= 128 has at most 8 significant bits: the BF16 is the FP32's top half
    for (int t = 0; t < 4; ++t) b[t] = __float_as_uint(static_cast<float>(slice_digit(X[t], Y[t], sl))) >> 16;
    *reinterpret_cast<uint2*>(out + kSliceK * sl + 4 * i) = make_uint2(b[0] | (b[1] << 16), b[2] | (b[3] << 16));
  }
}

// Generic-proxy writes (the digits) made visible to later TMA reads.
static __device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// The 72 MMAs of one tile (called by one thread): waits for its U tile (when
// it is a new one) and its V stage, then for each level L = i + j the digit
// pairs (i, j), both K halves of the 32 terms, into the level's 64 TMEM
// columns; the commit arrives on bar_acc once they are done (also when a wait
// ran out: then nothing was issued and the result is false).
static __device__ __forceinline__ bool tile_mmas(uint32_t tmem, uint32_t sA, uint32_t sB, uint32_t bar_a, bool wait_a,
                                                 uint32_t ph_a, uint32_t bar_b, uint32_t ph_b, uint32_t bar_acc) {
  bool ok = true;
  if (wait_a) ok = tm_wait(bar_a, ph_a & 1);
  ok = ok && tm_wait(bar_b, ph_b & 1);
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
          const uint64_t db = tm_desc(sB + (kbb / 64) * kUpdAtomB + (kbb % 64) * 2);
          tm_mma_f16(tmem + static_cast<uint32_t>((L - 2) * kUpdN), da, db, id, first ? 0 : 1);
          first = 0;
        }
      }
    }
  }
  tm_commit(bar_acc);
  return ok;
}

// W[r, c] += (U V)[r, c] for every r < n and every column c < n outside
// [kb, kb + jb), over the tiles [t_lo, t_hi) of this block (row-major order
// of the ceil(n / 128) x ceil(n / 64) tiles). dyn: this block's dynamic shared
// memory; err: the grid's error word.
static __device__ __noinline__ void sliced_update(SliceSmem& sm, unsigned char* dyn, const CUtensorMap* map_a,
                                                  const CUtensorMap* map_b, const SliceBufs& sb, double* W, int n,
                                                  int kb, int jb, int t_lo, int t_hi, int* err) {
  if (t_lo >= t_hi) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncb = (n + kUpdN - 1) / kUpdN;
  const uint32_t raw = su32(dyn);
  const uint32_t sA = (raw + 1023u) & ~1023u;
  const uint32_t sB[2] = {sA + kUpdABytes, sA + kUpdABytes + kUpdBBytes};
  double* Ts = reinterpret_cast<double*>(dyn + (sA - raw) + kUpdABytes + 2 * kUpdBBytes);  // [kUpdM][kUpdTsStride]
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
    fence_proxy_async_global();  // the digits other blocks wrote before the barrier, for the copies below
    issue(t_lo, true, 0);
    ++isA;
    ++isB[0];
  }
  if (tid == 32 && !tile_mmas(tmem, sA, sB[0], barA, true, phA, barB[0], phB[0], barAcc)) atomicExch(&sm.failed, 1);
  ++phA;
  ++phB[0];
  ++isAcc;
  bool failed = false;
  for (int t = t_lo; t < t_hi; ++t) {
    const int k = t - t_lo, st = k & 1;
    const int rb = t / ncb, cb = t % ncb;
    const int r0 = rb * kUpdM, c0 = cb * kUpdN;
    const bool has_next = t + 1 < t_hi;
    const bool next_new_a = has_next && ((t + 1) / ncb != rb);
    if (tid == 0 && has_next && !next_new_a) {  // the other V stage is free: its last reader was tile t - 1
      issue(t + 1, false, st ^ 1);
      ++isB[st ^ 1];
    }
    if (tid < kUpdN) sm.ecol[tid] = c0 + tid < n ? sb.bexp[c0 + tid] : 0;
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
    __syncthreads();  // the column exponents are in shared memory
    // levels -> exact dot products -> FP64, staged in Ts (warp w: TMEM lanes
    // 32 (w % 4) .. + 31 = tile rows, columns half (w / 4))
    if (acc_ok) {
      const int lrow = (warp & 3) * 32 + lane, half = warp >> 2;
      const int row = r0 + lrow;
      const int32_t er = row < n ? sb.aexp[row] : 0;
      for (int q = 0; q < 4; ++q) {
        const int cc = half * 32 + q * 8;
        uint32_t v[kSliceLevels][8];
        for (int L = 0; L < kSliceLevels; ++L)
          tm_ld8(tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + static_cast<uint32_t>(L * kUpdN + cc), v[L]);
        tm_ld_wait();
        for (int e = 0; e < 8; ++e) {
          int32_t c[kSliceLevels];
          for (int L = 0; L < kSliceLevels; ++L) c[L] = level_int(__uint_as_float(v[L][e]));
          Ts[lrow * kUpdTsStride + cc + e] = combine_levels_fp(c, er, sm.ecol[cc + e]);
        }
      }
    }
    tm_fence_before();
    __syncthreads();  // TMEM read, Ts complete
    // W += Ts: warp w takes rows w, w + 8, ..., lanes along the row
    // (coalesced). All 32 loads of a thread are issued before any store, so
    // their latencies overlap (the compiler may not move a load above a store
    // to memory it cannot prove distinct); the next tile's MMAs are issued
    // while these loads are in flight.
    constexpr int kPer = (kUpdM / 8) * 2;  // 16 rows x 2 column halves per thread
    double wv[kPer];
    if (acc_ok) {
#pragma unroll
      for (int it = 0; it < kPer; ++it) {
        const int rr = warp + 8 * (it >> 1), c = lane + 32 * (it & 1);
        const int gr = r0 + rr, gc = c0 + c;
        const bool ok = gr < n && gc < n && (gc < kb || gc >= kb + jb);
        wv[it] = ok ? __ldcg(W + (int64_t)gr * n + gc) : 0.0;
      }
    }
    if (has_next) {
      if (tid == 32 && sm.failed == 0 &&
          !tile_mmas(tmem, sA, sB[st ^ 1], barA, next_new_a, phA, barB[st ^ 1], phB[st ^ 1], barAcc))
        atomicExch(&sm.failed, 1);
      if (next_new_a) ++phA;
      ++phB[st ^ 1];
      ++isAcc;
    }
    if (acc_ok) {
#pragma unroll
      for (int it = 0; it < kPer; ++it) {
        const int rr = warp + 8 * (it >> 1), c = lane + 32 * (it & 1);
        const int gr = r0 + rr, gc = c0 + c;
        if (gr < n && gc < n && (gc < kb || gc >= kb + jb))
          W[(int64_t)gr * n + gc] = wv[it] + Ts[rr * kUpdTsStride + c];
      }
    }
    __syncthreads();  // Ts free for the next tile
    failed = sm.failed != 0;
    if (failed) break;
  }
  if (failed) {
    // wait (bounded) for this block's copies and MMAs still in flight: the
    // last phase issued on each barrier (a completed phase returns at once)
    if (tid == 0) {
      if (isA > sm.phase[0]) tm_wait(barA, (isA - 1) & 1);
      for (int s2 = 0; s2 < 2; ++s2)
        if (isB[s2] > sm.phase[1 + s2]) tm_wait(barB[s2], (isB[s2] - 1) & 1);
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
