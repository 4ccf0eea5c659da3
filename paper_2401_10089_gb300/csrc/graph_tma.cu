// graph_tma.cu -- precision form for uniform batches (every matrix n x n,
// including one large matrix): each graph product P_{j+2} = L_j R_j of the
// degree-optimal form (Sec. 3, eq. five_mult_degopt) in two launches.
//
//  k_graph_pack  forms the two factors L_j = sum_i h_{j,i} P_i and
//                R_j = sum_i g_{j,i} P_i once per element (FP32), splits them
//                into TF32 hi/lo or three BF16 slices and writes the slices in
//                the layout the tensor cores read: L_j row-major, R_j
//                transposed (both K-major), zero-padded to n_pad = 32 ceil(n/32).
//  k_graph_tma   streams 128 x KB tiles of those slices into shared memory
//                with TMA (cp.async.bulk.tensor.3d, 128-byte swizzle) through a
//                two-stage mbarrier pipeline: one thread issues the copies, one
//                thread issues tcgen05.mma (kind::tf32 or kind::f16) into an FP32
//                accumulator in TMEM, and the four warps read it back
//                (tcgen05.ld) for the epilogue (the output lin-comb, -2^s, the
//                balancing T L T^{-1}).
//
// Split products: TF32x3 hi*hi + hi*lo + lo*hi, BF16x3 the six s_a*s_b with
// a + b <= 2; the same arithmetic as k_graph_tc (graph_tc.cu), which serves
// ragged batches (where padding every matrix to n_max would waste memory).
// Every wait is bounded: a wait that runs out sets p.err and the block
// finishes without touching the output.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/logm.h"
#include "logm_internal.h"
#include "scheme_f32.cuh"
#include "tc_ptx.cuh"

namespace lg {

namespace {

constexpr int kTmM = 128;  // tile rows = TMEM lanes
constexpr int kTmThreads = 128;

template <int PREC>
struct TmCfg;
template <>
struct TmCfg<LOGM_PREC_TF32X3> {
  static constexpr int S = 2;     // slices per operand
  static constexpr int ESZ = 4;   // bytes per element
  static constexpr int KB = 32;   // K elements per stage (one 128-byte swizzle row)
  static constexpr int NB = 256;  // tile columns
  static constexpr int KSTEP = 8; // K per tcgen05.mma (32 bytes)
  static constexpr uint32_t FMT = 2;
};
template <>
struct TmCfg<LOGM_PREC_BF16X3> {
  static constexpr int S = 3;
  static constexpr int ESZ = 2;
  static constexpr int KB = 64;
  static constexpr int NB = 128;
  static constexpr int KSTEP = 16;
  static constexpr uint32_t FMT = 1;
};
constexpr int kTmStages = 2;

// Shared memory of k_graph_tma: per stage S slices of A (128 rows x 128 B)
// and S slices of B (NB rows x 128 B), each 1024-byte aligned (the 128-byte
// swizzle repeats every 8 rows = 1024 bytes). 96 KB per stage in both cases.
constexpr int kTmStageBytes = 96 * 1024;
constexpr size_t kTmSmemBytes = kTmStages * kTmStageBytes + 1024 /* barriers */ + 1024 /* alignment slack */;

static __device__ __forceinline__ bool tm_skip(const GraphParams& p, int b) {
  return p.info_dev && (p.info_dev[b] == 1 || p.info_dev[b] == 4);
}

template <int PREC>
static __device__ __forceinline__ void tm_mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, int acc) {
  if (PREC == LOGM_PREC_TF32X3)
    tm_mma_tf32(dt, a, b, id, acc);
  else
    tm_mma_f16(dt, a, b, id, acc);
}

static __device__ __forceinline__ uint32_t tm_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

static __device__ __forceinline__ void tm_geometry(const GraphParams& p, int b, int* n, int64_t* off) {
  if (p.n_uniform > 0) {
    *n = p.n_uniform;
    *off = (int64_t)b * p.n_uniform * p.n_uniform;
  } else {
    *n = p.n_dev[b];
    *off = p.off_dev[b];
  }
}

// ---------------------------------------------------------------------------
// Pack: factors of product j, split and laid out K-major for the tensor cores
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(256) k_graph_pack(GraphParams p, int n_pad) {
  using C = TmCfg<PREC>;
  __shared__ float tile[32][33];
  const int b = blockIdx.y;
  int n;
  int64_t off;
  tm_geometry(p, b, &n, &off);
  const int k = p.k_dev[b];
  if (tm_skip(p, b) || n < 1 || n > p.n_max || !needs_product(k, p.p3_given, p.j)) return;
  const int tiles_x = n_pad / 32;
  const int ty0 = (blockIdx.x / tiles_x) * 32, tx0 = (blockIdx.x % tiles_x) * 32;
  if (ty0 >= n_pad) return;
  Coeffs cf;
  scheme_coeffs(k, p.j, cf);
  const float* h = cf.h;
  const float* g = cf.g;
  const int terms = cf.terms;
  const int64_t nn_max = (int64_t)p.n_max * p.n_max;
  const float* P[6];
  for (int i = 0; i < 6; ++i) P[i] = p.gbuf + ((int64_t)b * 5 + (i < 4 ? i : 4)) * nn_max;
  const int64_t plane = (int64_t)n_pad * n_pad;
  unsigned char* A = static_cast<unsigned char*>(p.pack);
  unsigned char* B = A + (int64_t)p.count * C::S * plane * C::ESZ;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = ty0 + rr, c = tx0 + tx;
    float lv = 0.0f, rv = 0.0f;
    if (r < n && c < n) {
      const int64_t idx = (int64_t)r * n + c;
      for (int i = 0; i < terms; ++i) {
        const float v = P[i][idx];
        lv = fmaf(h[i], v, lv);
        rv = fmaf(g[i], v, rv);
      }
    }
    tile[rr][tx] = rv;
    const int64_t o = (int64_t)r * n_pad + c;
    if (PREC == LOGM_PREC_TF32X3) {
      const uint32_t hi = tm_tf32(lv);
      const uint32_t lo = tm_tf32(lv - __uint_as_float(hi));
      uint32_t* a = reinterpret_cast<uint32_t*>(A) + (int64_t)b * C::S * plane;
      a[o] = hi;
      a[plane + o] = lo;
    } else {
      const __nv_bfloat16 s0 = __float2bfloat16_rn(lv);
      const float r1 = lv - __bfloat162float(s0);
      const __nv_bfloat16 s1 = __float2bfloat16_rn(r1);
      const __nv_bfloat16 s2 = __float2bfloat16_rn(r1 - __bfloat162float(s1));
      __nv_bfloat16* a = reinterpret_cast<__nv_bfloat16*>(A) + (int64_t)b * C::S * plane;
      a[o] = s0;
      a[plane + o] = s1;
      a[2 * plane + o] = s2;
    }
  }
  __syncthreads();
  // R transposed: B[c][r] = R[r][c]
  for (int cc = ty; cc < 32; cc += 8) {
    const float rv = tile[tx][cc];
    const int64_t o = (int64_t)(tx0 + cc) * n_pad + (ty0 + tx);
    if (PREC == LOGM_PREC_TF32X3) {
      const uint32_t hi = tm_tf32(rv);
      const uint32_t lo = tm_tf32(rv - __uint_as_float(hi));
      uint32_t* bb = reinterpret_cast<uint32_t*>(B) + (int64_t)b * C::S * plane;
      bb[o] = hi;
      bb[plane + o] = lo;
    } else {
      const __nv_bfloat16 s0 = __float2bfloat16_rn(rv);
      const float r1 = rv - __bfloat162float(s0);
      const __nv_bfloat16 s1 = __float2bfloat16_rn(r1);
      const __nv_bfloat16 s2 = __float2bfloat16_rn(r1 - __bfloat162float(s1));
      __nv_bfloat16* bb = reinterpret_cast<__nv_bfloat16*>(B) + (int64_t)b * C::S * plane;
      bb[o] = s0;
      bb[plane + o] = s1;
      bb[2 * plane + o] = s2;
    }
  }
}

// ---------------------------------------------------------------------------
// The product: TMA -> shared memory -> tcgen05.mma -> TMEM -> epilogue
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(kTmThreads, 1)
    k_graph_tma(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, GraphParams p,
                int n_pad, int nbox) {
  using C = TmCfg<PREC>;
  extern __shared__ unsigned char tm_smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  const uint32_t raw = su32(tm_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sbase = tm_smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + kTmStages * kTmStageBytes);  // full[2], empty[2], accum
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);

  const int b = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int n;
  int64_t off;
  tm_geometry(p, b, &n, &off);
  const int k = p.k_dev[b];
  if (tm_skip(p, b) || n < 1 || n > p.n_max || !needs_product(k, p.p3_given, p.j)) return;
  const int n_tiles = (n_pad + nbox - 1) / nbox;
  const int m_tiles = (n + kTmM - 1) / kTmM;
  if ((int)blockIdx.x >= m_tiles * n_tiles) return;
  const int r0 = (blockIdx.x / n_tiles) * kTmM;
  const int c0 = (blockIdx.x % n_tiles) * nbox;
  if (c0 >= n) return;
  const int ncols = nbox <= 32 ? 32 : (nbox <= 64 ? 64 : (nbox <= 128 ? 128 : 256));

  const uint32_t full0 = su32(&bars[0]), empty0 = su32(&bars[2]), accum = su32(&bars[4]);
  if (tid == 0) {
    for (int t = 0; t < 5; ++t) tm_bar_init(su32(&bars[t]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int a_bytes = kTmM * 128;          // one A slice per stage
  const int b_bytes = nbox * 128;          // one B slice per stage (nbox rows of 128 B)
  const int b_stride = C::NB * 128;        // B slice slot size
  const uint32_t stage_tx = (uint32_t)(C::S * (a_bytes + b_bytes));
  const int kchunks = (n + C::KB - 1) / C::KB;
  __shared__ int s_failed;
  if (tid == 0) s_failed = 0;
  __syncthreads();

  if (warp == 0 && lane == 0) {
    // producer: TMA copies of stage kc (all slices of both operands)
    for (int kc = 0; kc < kchunks; ++kc) {
      const int st = kc & 1;
      if (kc >= 2 && !tm_wait(empty0 + 8 * st, ((kc >> 1) - 1) & 1)) {
        s_failed = 1;
        break;
      }
      const uint32_t sa = base + st * kTmStageBytes;
      const uint32_t sb = sa + C::S * a_bytes;
      tm_expect(full0 + 8 * st, stage_tx);
      for (int s = 0; s < C::S; ++s) {
        tm_load3d(sa + s * a_bytes, &ta, full0 + 8 * st, kc * C::KB, r0, b * C::S + s);
        tm_load3d(sb + s * b_stride, &tb, full0 + 8 * st, kc * C::KB, c0, b * C::S + s);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id = tm_idesc(C::FMT, kTmM, nbox);
    int first = 1;
    for (int kc = 0; kc < kchunks; ++kc) {
      const int st = kc & 1;
      if (!tm_wait(full0 + 8 * st, (kc >> 1) & 1)) {
        s_failed = 1;
        break;
      }
      tm_fence_after();
      const uint32_t sa = base + st * kTmStageBytes;
      const uint32_t sb = sa + C::S * a_bytes;
      for (int ks = 0; ks < C::KB / C::KSTEP; ++ks) {
        const uint32_t koff = ks * C::KSTEP * C::ESZ;  // 32 bytes per step inside the swizzle row
        for (int ia = 0; ia < C::S; ++ia)
          for (int ib = 0; ib < C::S; ++ib) {
            if (ia + ib > C::S - 1) continue;  // TF32x3: (0,0) (0,1) (1,0); BF16x3: a + b <= 2
            const uint64_t da = tm_desc(sa + ia * a_bytes + koff);
            const uint64_t db = tm_desc(sb + ib * b_stride + koff);
            tm_mma<PREC>(tmem, da, db, id, first ? 0 : 1);
            first = 0;
          }
      }
      tm_commit(empty0 + 8 * st);
    }
    tm_commit(accum);
  }
  __syncwarp();
  // epilogue: all four warps wait for the accumulator
  const bool ok = tm_wait(accum, 0);
  tm_fence_after();
  __syncthreads();
  const int failed = s_failed || !ok;
  if (!failed) {
    const int row = r0 + warp * 32 + lane;
    const int last = is_last_product(k, p.j);
    const float scale = (last && p.s_dev) ? -ldexpf(1.0f, p.s_dev[b]) : 1.0f;
    float yv[6] = {0, 0, 0, 0, 0, 0};
    float ylast = 0.0f;
    if (last) {
      for (int i = 0; i <= p.j - 1 && i < 5; ++i) yv[i] = scheme_y(k, i);
      ylast = scheme_y(k, p.j);
    }
    const int64_t nn_max = (int64_t)p.n_max * p.n_max;
    const float* P[6];
    for (int i = 0; i < 6; ++i) P[i] = p.gbuf + ((int64_t)b * 5 + (i < 4 ? i : 4)) * nn_max;
    float* outP = p.gbuf + ((int64_t)b * 5 + (p.j < 4 ? p.j : 4)) * nn_max;  // P_{j+2} slot
    const double* bal = p.bal ? p.bal + (int64_t)b * p.n_max : nullptr;
    for (int cb = 0; cb < nbox; cb += 8) {
      uint32_t r[8];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(cb);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < n) {
        for (int t = 0; t < 8; ++t) {
          const int gc = c0 + cb + t;
          if (gc >= n) break;
          const float acc = __uint_as_float(r[t]);
          const int64_t idx = (int64_t)row * n + gc;
          if (!last) {
            outP[idx] = acc;
          } else {
            float v = ylast * acc;
            for (int i = 0; i < p.j && i < 5; ++i) v = fmaf(yv[i], P[i][idx], v);
            v *= scale;
            if (bal) v *= (float)(bal[row] / bal[gc]);
            if (p.out_dtype == 0)
              static_cast<double*>(p.L)[off + idx] = static_cast<double>(v);
            else
              static_cast<float*>(p.L)[off + idx] = v;
          }
        }
      }
    }
  } else if (tid == 0 && p.err) {
    atomicExch(p.err, 1);
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Host side: tensor maps (the encoder is taken from the driver at run time)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  // the driver's entry point is the same for every device; looked up once
  // (a function-local static is initialised once even with several threads)
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(f);
    return static_cast<EncodeTiledFn>(nullptr);
  }();
  return fn;
}

// 3-D map over count * S planes of n_pad x n_pad elements, box KB x rows x 1,
// 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* m, void* base, int prec, int n_pad, int planes, int box_rows) {
  EncodeTiledFn f = encoder();
  if (!f) return false;
  const bool tf = prec == LOGM_PREC_TF32X3;
  const int esz = tf ? 4 : 2;
  const cuuint64_t dims[3] = {(cuuint64_t)n_pad, (cuuint64_t)n_pad, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)n_pad * esz, (cuuint64_t)n_pad * n_pad * esz};
  const cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = f(m, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int PREC>
cudaError_t run_tma(const GraphParams& p, cudaStream_t st) {
  using C = TmCfg<PREC>;
  const int n = p.n_max;  // uniform batch: n_max == n
  const int n_pad = (n + 31) / 32 * 32;
  const int nbox = n_pad < C::NB ? n_pad : C::NB;
  const int planes = p.count * C::S;
  unsigned char* A = static_cast<unsigned char*>(p.pack);
  unsigned char* B = A + (size_t)planes * n_pad * n_pad * C::ESZ;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, PREC, n_pad, planes, kTmM)) return cudaErrorNotSupported;
  if (!make_map(&tb, B, PREC, n_pad, planes, nbox)) return cudaErrorNotSupported;
  static DeviceOnce attr;
  cudaError_t ea = attr.run([] {
    return cudaFuncSetAttribute(k_graph_tma<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmSmemBytes);
  });
  if (ea != cudaSuccess) return ea;
  const int tiles = ((n + kTmM - 1) / kTmM) * ((n_pad + nbox - 1) / nbox);
  const dim3 pgrid((n_pad / 32) * (n_pad / 32), p.count);
  for (int j = 1; j <= 5; ++j) {
    GraphParams q = p;
    q.j = j;
    k_graph_pack<PREC><<<pgrid, 256, 0, st>>>(q, n_pad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_graph_tma<PREC><<<dim3(tiles, p.count), kTmThreads, kTmSmemBytes, st>>>(ta, tb, q, n_pad, nbox);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

// Bytes of the packed slices for a uniform batch (both operands, the larger
// of the two precisions: TF32 2 x 4 bytes, BF16 3 x 2 bytes per element).
size_t graph_pack_bytes(int count, int n) {
  const size_t n_pad = (size_t)(n + 31) / 32 * 32;
  return 2 * (size_t)count * n_pad * n_pad * 8;
}

cudaError_t launch_graph_tma(const GraphParams& p, cudaStream_t st) {
  if (p.count <= 0) return cudaSuccess;
  return p.precision == LOGM_PREC_TF32X3 ? run_tma<LOGM_PREC_TF32X3>(p, st) : run_tma<LOGM_PREC_BF16X3>(p, st);
}

}  // namespace lg
