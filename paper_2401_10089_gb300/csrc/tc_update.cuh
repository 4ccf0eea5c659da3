// tc_update.cuh -- the rank-K updates of the whole-GPU kernel,
// W[:, cols] += U V, on the tensor cores with FP64 accuracy.
//
// U (n x K) and V (K x n), K = 32 nc for nc <= kMaxChunks chunks, are split
// into exact BF16 digits (fp64_slices.cuh): every row of U and every column
// of V gets one power-of-two scale over its K values and eight digits per
// value, stored K-major in global memory (kDigRow BF16 per row or column:
// chunk c at kChunkDig c; inside a chunk the half h of its 32 terms at 128 h,
// digit s of that half at 16 s). Each block then runs its share of the
// 128 x 64 output tiles of W:
//   * thread 0 streams the digits through a ring of kUpdStages shared-memory
//     stages with TMA, one stage per (chunk, half): 128 x 128 BF16 of U (one
//     3-D copy: two 128-byte swizzle atoms of 4 digits x 16 terms per row)
//     and 64 x 128 of V (one 3-D copy, 32-byte swizzle: per digit its 64
//     columns, stacked as 512 operand rows);
//   * thread 32 issues, per stage, 12 tcgen05.mma (kind::f16, BF16 x BF16 ->
//     FP32, M = 128, K = 16): digit i of U against the digits j = 1 .. 9 - i
//     of V in pieces of up to four (N = 64 per digit, up to 256), written at
//     TMEM column 64 (i + j - 2), so that the pair (i, j) lands in the 64
//     columns of its level L = i + j (8 levels = all 512 columns),
//     accumulated over all stages of the tile. A level sum is an integer of
//     magnitude <= nc 2^22 <= 2^24, so FP32 accumulation is exact;
//   * all eight warps read the levels back (tcgen05.ld), combine them into the
//     exact integer dot product and round it to FP64 into a shared-memory
//     tile; then the next tile's copies and MMAs run (threads 0 and 32)
//     while warps 2 .. 7 add the staged tile to W row by row (coalesced).
// Per element that is four FP64 instructions (conversion and addition) for K
// terms instead of K FP64 FMAs.
//
// Every mbarrier wait is bounded (kTmWaitLimit polls); a wait that runs out
// sets the grid's error word, and the kernel reports LOGM_INFO_TIMEOUT for the
// matrix instead of hanging.
#pragma once

#include <cuda_bf16.h>

#include "fp64_slices.cuh"
#include "tc_ptx.cuh"

namespace lg {

constexpr int kUpdM = 128, kUpdN = 64;                       // output tile of W: rows x columns
constexpr int kMaxChunks = 4;                                // K of one update: up to 4 x 32 terms
constexpr int kChunkDig = kSlices * kSliceK;                 // digits of one chunk of a row: 256 BF16
constexpr int kDigRow = kMaxChunks * kChunkDig;              // digit buffer row: 1024 BF16
constexpr int kUpdStages = 3;                                // TMA ring depth
constexpr uint32_t kAtomA = kUpdM * 128;       // U: one 128-byte swizzle box (4 digits x 16 terms per row)
constexpr uint32_t kDigB = kUpdN * 32;          // V: one digit of 16 terms for 64 columns (32-byte swizzle)
constexpr uint32_t kStageA = 2 * kAtomA, kStageB = kSlices * kDigB;  // half a chunk: 32 KB + 16 KB
constexpr uint32_t kStageBytes = kStageA + kStageB;
constexpr int kUpdTsStride = kUpdN + 1;                      // staged tile: doubles per row (padded)
constexpr uint32_t kUpdTsBytes = kUpdM * kUpdTsStride * 8;   // 65 KB
constexpr size_t kUpdSmemBytes = kUpdStages * kStageBytes + kUpdTsBytes + 1024;  // + alignment slack
constexpr int kUpdTmemCols = kSliceLevels * kUpdN;           // 512
static_assert(kUpdTmemCols == 512, "eight levels of 64 columns fill TMEM");
static_assert(kSlices == 8, "a stage holds two swizzle boxes of four digits");

// Tensor maps of the digit buffers, per inversion group, 3-D views of the
// n_max x kDigRow BF16 buffers: U as (64 terms, row, 64-term group) with
// boxes 64 x 128 x 2, 128-byte swizzle; V as (16 terms, column, 16-term
// group) with boxes 16 x 64 x 8, 32-byte swizzle.
struct SliceMaps {
  CUtensorMap a[2];
  CUtensorMap b[2];
};

struct SliceBufs {
  __nv_bfloat16* adig;  // [n_max][kDigRow]: digits of the rows of U
  __nv_bfloat16* bdig;  // [n_max][kDigRow]: digits of the columns of V
  int32_t* aexp;        // [n_max] scale exponent of each row of U
  int32_t* bexp;        // [n_max] scale exponent of each column of V
};

// Barriers and lifetime counters of the engine (they persist across calls:
// a stage with lifetime index u uses ring slot u % kUpdStages for the
// (u / kUpdStages)-th time, which fixes the phase parity of its barriers).
struct SliceSmem {
  unsigned long long full[kUpdStages];   // stage loaded (TMA transaction bytes)
  unsigned long long empty[kUpdStages];  // stage's MMAs done (tcgen05.commit)
  unsigned long long acc;                // tile's MMAs done
  uint32_t stages;                       // stages loaded and consumed so far
  uint32_t tiles;                        // tiles accumulated so far
  uint32_t tmem;                         // TMEM base address of the level accumulators
  int32_t ecol[kUpdN];                   // scale exponents of the current tile's columns of V
};

// Which tiles and columns of W an update touches: output column tiles
// cb0 .. cb0 + ncbt - 1 of every row tile, those from gap_at on shifted by
// gap (so that [gap_at, gap_at + gap) is skipped), and within them every
// column outside [mk, mk + mj).
struct UpdTiles {
  int nc;
  int cb0, ncbt, gap_at, gap;
  int mk, mj;
};

// The digits of one row of up to 32 NC values split among the 8 lanes of an
// aligned lane group (lanes 8q .. 8q + 7 of a warp): lane i holds, for every
// chunk c < NC, the values k = 4 i .. 4 i + 3 of that chunk in v[4 c .. 4 c + 3]
// (zero past the row's length). The group forms the row's scale exponent (the
// largest magnitude by integer comparison of the bit patterns: NaN above Inf
// above every finite value), each lane the fixed-point integers and all eight
// digits of its values, and writes them as 8-byte pieces of the row at out
// (chunks c < nc); lane 0 stores the exponent at *eo. Every lane of the warp
// must call this (the shuffles); `valid` lanes store.
template <int NC>
static __device__ __forceinline__ void slice_row8(const double* v, int i, bool valid, int nc, __nv_bfloat16* out,
                                                  int32_t* eo) {
  unsigned long long mb = 0;
#pragma unroll
  for (int t = 0; t < 4 * NC; ++t) {
    const unsigned long long a = lg_dbits(v[t]) & 0x7FFFFFFFFFFFFFFFull;
    mb = a > mb ? a : mb;
  }
#pragma unroll
  for (int x = 1; x < 8; x <<= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, mb, x);
    mb = o > mb ? o : mb;
  }
  const int32_t e = slice_exponent(lg_bitsd(mb));
  if (valid && i == 0) *eo = e;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    int64_t X[4];
    uint64_t Y[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      X[t] = e != kSliceNonFinite ? slice_fixed_int(v[4 * c + t], e) : 0;
      Y[t] = slice_bias(X[t]);
    }
    if (valid && c < nc) {
      __nv_bfloat16* o = out + kChunkDig * c + 128 * (i >> 2) + 4 * (i & 3);
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) {
        uint32_t b[4];
        // |d| <= 128 has at most 8 significant bits: the BF16 is the FP32's top half
#pragma unroll
        for (int t = 0; t < 4; ++t) b[t] = __float_as_uint(static_cast<float>(slice_digit(X[t], Y[t], sl))) >> 16;
        *reinterpret_cast<uint2*>(o + 16 * sl) = make_uint2(b[0] | (b[1] << 16), b[2] | (b[3] << 16));
      }
    }
  }
}

// One row of 32 values (one chunk), out of line: the split of the Gauss-Jordan
// panels and pivot rows.
static __device__ __noinline__ void slice_row8_1(double v0, double v1, double v2, double v3, int i, bool valid,
                                                 __nv_bfloat16* out, int32_t* eo) {
  const double v[4] = {v0, v1, v2, v3};
  slice_row8<1>(v, i, valid, 1, out, eo);
}

// Generic-proxy writes (the digits) made visible to later TMA reads.
static __device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Thread 0: loads stage s of a tile (chunk s / 2, half s % 2) of row tile rb
// and column tile cb into ring slot u % kUpdStages, u the stage's lifetime
// index, once the slot's previous MMAs are done. False when that wait ran out.
static __device__ __forceinline__ bool upd_produce(SliceSmem& sm, uint32_t ring, const CUtensorMap* map_a,
                                                   const CUtensorMap* map_b, uint32_t u, int rb, int cb, int s) {
  const uint32_t slot = u % kUpdStages, use = u / kUpdStages;
  if (use > 0 && !tm_wait(su32(&sm.empty[slot]), (use - 1) & 1)) return false;
  const uint32_t fb = su32(&sm.full[slot]);
  const uint32_t sA = ring + slot * kStageBytes, sB = sA + kStageA;
  const int x = kChunkDig * (s >> 1) + 128 * (s & 1);
  tm_expect(fb, kStageBytes);
  tm_load3d(sA, map_a, fb, 0, rb * kUpdM, x / 64);
  tm_load3d(sB, map_b, fb, 0, cb * kUpdN, x / 16);
  return true;
}

// Thread 0: stages [s_from, s_to) of the tile whose first stage has lifetime
// index u0; *done counts the stages issued.
static __device__ __noinline__ bool upd_produce_range(SliceSmem& sm, uint32_t ring, const CUtensorMap* map_a,
                                                      const CUtensorMap* map_b, uint32_t u0, int rb, int cb,
                                                      int s_from, int s_to, uint32_t* done) {
  for (int s = s_from; s < s_to; ++s) {
    if (!upd_produce(sm, ring, map_a, map_b, u0 + s, rb, cb, s)) return false;
    ++*done;
  }
  return true;
}

// Thread 32: the MMAs of a tile, stage by stage as they arrive: per stage (a
// half chunk) and digit i of U, digit i against the digits j = 1 .. 9 - i of
// V in pieces of up to four (one MMA each, N = 64 per digit) at TMEM column
// 64 (i + j - 2): 12 MMAs covering the 36 pairs of levels 2 .. 9. In the
// tile's first stage the two pieces of digit 1 write every level once and
// start the sums (no accumulate); every other MMA accumulates. Each stage's
// commit frees its slot; the final commit arrives on acc once all are done
// (also after a wait ran out, so that the readers are released; the result is
// then false).
static __device__ __noinline__ bool upd_mma_tile(SliceSmem& sm, uint32_t ring, uint32_t tmem, uint32_t u0, int S2) {
  bool ok = true;
  for (int s = 0; s < S2 && ok; ++s) {
    const uint32_t u = u0 + s, slot = u % kUpdStages, use = u / kUpdStages;
    ok = tm_wait(su32(&sm.full[slot]), use & 1);
    if (!ok) break;
    tm_fence_after();
    const uint32_t sA = ring + slot * kStageBytes, sB = sA + kStageA;
#pragma unroll
    for (int i = 1; i <= kSlices; ++i) {
      const uint64_t da = tm_desc(sA + ((i - 1) >> 2) * kAtomA + ((i - 1) & 3) * 32);
#pragma unroll
      for (int j0 = 1; j0 <= kSlices + 1 - i; j0 += 4) {
        const int cnt = (kSlices + 2 - i - j0) < 4 ? (kSlices + 2 - i - j0) : 4;
        const uint64_t db = tm_desc_sw32(sB + (j0 - 1) * kDigB);
        tm_mma_f16(tmem + static_cast<uint32_t>((i + j0 - 2) * kUpdN), da, db, tm_idesc(1, kUpdM, kUpdN * cnt),
                   (s == 0 && i == 1) ? 0 : 1);
      }
    }
    tm_commit(su32(&sm.empty[slot]));
  }
  tm_commit(su32(&sm.acc));
  return ok;
}

// W[r, c] += (U V)[r, c] over the tiles [t_lo, t_hi) of this block (row-major
// order of the ceil(n / 128) x ut.ncbt tiles that ut names), every r < n and
// every column c < n of those tiles outside [ut.mk, ut.mk + ut.mj). dyn: this
// block's dynamic shared memory; err: the grid's error word.
static __device__ __noinline__ void sliced_update(SliceSmem& sm, unsigned char* dyn, const CUtensorMap* map_a,
                                                  const CUtensorMap* map_b, const SliceBufs& sb, double* W, int n,
                                                  const UpdTiles ut, int t_lo, int t_hi, int* err) {
  if (t_lo >= t_hi) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S2 = 2 * ut.nc;                               // stages per tile
  const int npre = S2 < kUpdStages ? S2 : kUpdStages;     // stages of the next tile loaded ahead
  const uint32_t raw = su32(dyn);
  const uint32_t ring = (raw + 1023u) & ~1023u;
  double* Ts = reinterpret_cast<double*>(dyn + (ring - raw) + kUpdStages * kStageBytes);  // [kUpdM][kUpdTsStride]
  const uint32_t u_base = sm.stages, tile_base = sm.tiles, tmem = sm.tmem;
  const uint32_t bar_acc = su32(&sm.acc);
  __syncthreads();  // everyone has read the counters
  auto tile_of = [&](int t, int* rb, int* cb) {
    *rb = t / ut.ncbt;
    int c = ut.cb0 + t % ut.ncbt;
    if (c >= ut.gap_at) c += ut.gap;
    *cb = c;
  };
  bool bad = false;         // this thread saw a wait run out
  uint32_t produced = 0;    // thread 0: stages issued
  uint32_t committed = 0;   // thread 32: tiles committed
  {
    int rb, cb;
    tile_of(t_lo, &rb, &cb);
    if (tid == 0) bad = !upd_produce_range(sm, ring, map_a, map_b, u_base, rb, cb, 0, S2, &produced);
    if (tid == 32) {
      bad = !upd_mma_tile(sm, ring, tmem, u_base, S2);
      ++committed;
    }
  }
  int fail = 0, done_tiles = 0;
  for (int t = t_lo; t < t_hi; ++t) {
    const int k = t - t_lo;
    int rb, cb, nrb = 0, ncb = 0;
    tile_of(t, &rb, &cb);
    const int r0 = rb * kUpdM, c0 = cb * kUpdN;
    const bool has_next = t + 1 < t_hi;
    if (has_next) tile_of(t + 1, &nrb, &ncb);
    const uint32_t u_next = u_base + static_cast<uint32_t>((k + 1) * S2);
    if (tid < kUpdN) sm.ecol[tid] = c0 + tid < n ? sb.bexp[c0 + tid] : 0;
    // tcgen05.ld is warp-collective: a warp reads the accumulators only if all its lanes saw them ready
    const bool acc_ok = __all_sync(0xffffffffu, tm_wait(bar_acc, (tile_base + k) & 1));
    tm_fence_after();
    bad = bad || !acc_ok;
    // the ring is free (all of this tile's MMAs are done): the next tile's first stages
    if (tid == 0 && has_next && !bad)
      bad = !upd_produce_range(sm, ring, map_a, map_b, u_next, nrb, ncb, 0, npre, &produced);
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
        // a level sum above 2^22 (possible for K > 32 only) needs the two-part
        // conversion: one vote per warp and column group picks the loop
        bool wide = false;
        if (ut.nc > 1)
          for (int L = 0; L < kSliceLevels; ++L)
            for (int e = 0; e < 8; ++e) wide |= fabsf(__uint_as_float(v[L][e])) > 4194304.0f;
        if (__any_sync(0xffffffffu, wide)) {
          for (int e = 0; e < 8; ++e) {
            int32_t c[kSliceLevels];
            for (int L = 0; L < kSliceLevels; ++L) c[L] = level_int_wide(__uint_as_float(v[L][e]));
            Ts[lrow * kUpdTsStride + cc + e] = combine_levels_fp(c, er, sm.ecol[cc + e]);
          }
        } else {
          // branch-free for every element; the rare ones (a non-finite row or
          // column, a subnormal or overflowing result) again through the full route
          bool slow = false;
          for (int e = 0; e < 8; ++e) {
            int32_t c[kSliceLevels];
            for (int L = 0; L < kSliceLevels; ++L) c[L] = level_int(__uint_as_float(v[L][e]));
            bool sl;
            Ts[lrow * kUpdTsStride + cc + e] = combine_levels_fast(c, er, sm.ecol[cc + e], &sl);
            slow = slow || sl;
          }
          if (__any_sync(0xffffffffu, slow) && slow)
            for (int e = 0; e < 8; ++e) {
              int32_t c[kSliceLevels];
              for (int L = 0; L < kSliceLevels; ++L) c[L] = level_int(__uint_as_float(v[L][e]));
              Ts[lrow * kUpdTsStride + cc + e] = combine_levels_fp(c, er, sm.ecol[cc + e]);
            }
        }
      }
    }
    tm_fence_before();
    __syncthreads();  // TMEM read, Ts complete
    // W += Ts: warp w = 2 .. 7 takes rows w - 2, w + 4, ..., lanes along the
    // row (coalesced). All loads of a thread are issued before any store, so
    // their latencies overlap (the compiler may not move a load above a store
    // to memory it cannot prove distinct); meanwhile thread 0 loads the next
    // tile's remaining stages and thread 32 issues its MMAs.
    constexpr int kWW = 6;                                   // warps on W
    constexpr int kPer = 2 * ((kUpdM + kWW - 1) / kWW);      // rows x 2 column halves per thread
    const int ww = warp - (8 - kWW);
    double wv[kPer];
    if (acc_ok && ww >= 0) {
#pragma unroll
      for (int it = 0; it < kPer; ++it) {
        const int rr = ww + kWW * (it >> 1), c = lane + 32 * (it & 1);
        const int gr = r0 + rr, gc = c0 + c;
        const bool ok = rr < kUpdM && gr < n && gc < n && (gc < ut.mk || gc >= ut.mk + ut.mj);
        wv[it] = ok ? __ldcg(W + (int64_t)gr * n + gc) : 0.0;
      }
    }
    if (has_next && !bad) {
      if (tid == 0) bad = !upd_produce_range(sm, ring, map_a, map_b, u_next, nrb, ncb, npre, S2, &produced);
      if (tid == 32) {
        bad = !upd_mma_tile(sm, ring, tmem, u_next, S2);
        ++committed;
      }
    }
    if (acc_ok && ww >= 0) {
#pragma unroll
      for (int it = 0; it < kPer; ++it) {
        const int rr = ww + kWW * (it >> 1), c = lane + 32 * (it & 1);
        const int gr = r0 + rr, gc = c0 + c;
        if (rr < kUpdM && gr < n && gc < n && (gc < ut.mk || gc >= ut.mk + ut.mj))
          W[(int64_t)gr * n + gc] = wv[it] + Ts[rr * kUpdTsStride + c];
      }
    }
    ++done_tiles;
    fail = __syncthreads_or(bad ? 1 : 0);  // also: Ts free for the next tile
    if (fail) break;
  }
  if (fail) {
    // wait (bounded) for this block's copies and MMAs still in flight: the
    // last stages issued (each the latest use of its slot) and the last
    // tile committed, then report the failure
    if (tid == 32) sm.ecol[0] = static_cast<int32_t>(committed);
    __syncthreads();
    if (tid == 0) {
      const uint32_t last = static_cast<uint32_t>(sm.ecol[0]);
      const uint32_t first = produced > kUpdStages ? produced - kUpdStages : 0;
      for (uint32_t p = first; p < produced; ++p) {
        const uint32_t u = u_base + p;
        tm_wait(su32(&sm.full[u % kUpdStages]), (u / kUpdStages) & 1);
      }
      if (last > 0) tm_wait(bar_acc, (tile_base + last - 1) & 1);
      atomicExch(err, 1);
    }
  }
  if (tid == 0) {
    // lifetime counts (after a failure they no longer matter: the kernel
    // skips every later update)
    sm.stages = u_base + static_cast<uint32_t>(done_tiles * S2);
    sm.tiles = tile_base + static_cast<uint32_t>(done_tiles);
  }
  __syncthreads();
}

}  // namespace lg
