// graph_tc.cu -- the computation-graph products (Sec. 3, eq. five_mult_degopt)
// of the precision form on the 5th-generation tensor cores (tcgen05, TMEM
// accumulators).
//
// After the FP64 stage (plan and square roots) hands over P_2 = X and
// P_3 = X^2 in FP32, every product P_{j+2} = (sum_i h_{j,i} P_i)(sum_i g_{j,i} P_i)
// of a batch runs in one launch: a block owns a 128 x N tile of one matrix's
// product, forms the two lin-comb factors in FP32 while staging them, splits
// each value into tensor-core slices and accumulates the slice products in
// FP32 in TMEM:
//   TF32x3 : a = hi + lo (TF32),        hi*hi + hi*lo + lo*hi        (kind::tf32)
//   BF16x3 : a = a0 + a1 + a2 (BF16),   the 6 slice products i+j <= 2 (kind::f16)
// The last product's epilogue applies the output lin-comb z = sum_i y_i P_i and
// the scale -2^s, and writes L. No FP64 arithmetic runs in this file: on GB300
// FP64 is ~2000x slower than the tensor cores, so even the O(n^2) lin-combs
// would dominate.
//
// Operands are staged in shared memory in the canonical K-major, no-swizzle
// layout: 8-row x 16-byte core matrices, core (group g, k-core c) at
// g * SBO + c * 128 bytes, rows 16 bytes apart inside a core. One MMA covers
// 32 bytes of K (two cores), so its descriptor starts 256 bytes further per
// K step. One thread issues the MMAs; completion is tracked with an mbarrier
// (tcgen05.commit). Every wait is bounded: on time-out the block records an
// error, still frees its TMEM, and returns.
#include <cstdint>
#include <cuda_bf16.h>

#include "../../include/logm.h"
#include "logm_internal.h"
#include "scheme_f32.cuh"

namespace lg {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;      // rows per tile (MMA M)
constexpr int kTcN = 256;      // max columns per tile (MMA N)
constexpr int kTcK = 32;       // K elements staged per round
constexpr long long kTcWaitLimit = 1ll << 20;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle.
static __device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format `fmt` (1 BF16,
// 2 TF32), both K-major, M x N.
static __device__ __forceinline__ uint32_t idesc(uint32_t fmt, int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= fmt << 7;
  d |= fmt << 10;
  d |= static_cast<uint32_t>(N >> 3) << 17;
  d |= static_cast<uint32_t>(M >> 4) << 24;
  return d;
}

static __device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

static __device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

static __device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

static __device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

static __device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

static __device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
static __device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------------------
// The batched product kernel
// ---------------------------------------------------------------------------
struct TcSmem {
  // operand slices, K-major no-swizzle; sized for the larger (TF32x3) case:
  // A: 2 slices x 128 rows x 128 B, B: 2 slices x 256 rows x 128 B
  alignas(1024) unsigned char a[2 * kTcM * 128];
  alignas(1024) unsigned char b[2 * kTcN * 128];
  alignas(8) unsigned long long mbar;
  uint32_t tmem_base;
  int skip;
};

template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 1) k_graph_tc(GraphParams p) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(tc_smem_raw);
  const int b = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int n;
  int64_t off;
  if (p.n_uniform > 0) {
    n = p.n_uniform;
    off = (int64_t)b * n * n;
  } else {
    n = p.n_dev[b];
    off = p.off_dev[b];
  }
  const int k = p.k_dev[b];
  if (p.info_dev && (p.info_dev[b] == 1 || p.info_dev[b] == 4)) return;  // no result (singular, non-finite)
  if (n < 1 || n > p.n_max || !needs_product(k, p.p3_given, p.j)) return;
  const int n_pad = ((n + 15) / 16) * 16;
  const int n_tiles = (n_pad + kTcN - 1) / kTcN;
  const int m_tiles = (n + kTcM - 1) / kTcM;
  if ((int)blockIdx.x >= m_tiles * n_tiles) return;
  const int r0 = (blockIdx.x / n_tiles) * kTcM;
  const int c0 = (blockIdx.x % n_tiles) * kTcN;
  const int N = min(kTcN, n_pad - c0);  // multiple of 16, 16..256
  int ncols = 32;
  while (ncols < N) ncols <<= 1;

  const int64_t nn_max = (int64_t)p.n_max * p.n_max;
  const float* P[6];
  for (int i = 0; i < 6; ++i) P[i] = p.gbuf + ((int64_t)b * 5 + min(i, 4)) * nn_max;  // P_2 .. P_6
  Coeffs cf;
  scheme_coeffs(k, p.j, cf);

  const uint32_t mbar = smem_u32(&S.mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem_base;

  // slice geometry (bytes): TF32 4 elements per 16-byte core row, BF16 8
  constexpr int esz = (PREC == LOGM_PREC_TF32X3) ? 4 : 2;
  constexpr int epc = 16 / esz;                 // elements per core row
  constexpr int sbo = (kTcK / epc) * 128;       // bytes per 8-row group of one slice
  const int a_slice = (kTcM / 8) * sbo;
  const int b_slice = (kTcN / 8) * sbo;
  const uint32_t id = idesc(PREC == LOGM_PREC_TF32X3 ? 2u : 1u, kTcM, N);

  int failed = 0;
  uint32_t phase = 0;
  const int kchunks = (n + kTcK - 1) / kTcK;
  for (int kc = 0; kc < kchunks; ++kc) {
    const int k0 = kc * kTcK;
    // A tile: rows r0..r0+127, K k0..k0+31: lin-comb sum_i h_i P_i, then split
    for (int e = tid; e < kTcM * kTcK; e += kTcThreads) {
      const int rr = e / kTcK, kk = e % kTcK;
      const int gr = r0 + rr, gk = k0 + kk;
      float v = 0.0f;
      if (gr < n && gk < n) {
        const int64_t idx = (int64_t)gr * n + gk;
        for (int i = 0; i < cf.terms; ++i) v = fmaf(cf.h[i], P[i][idx], v);
      }
      const int byte = (rr >> 3) * sbo + (kk / epc) * 128 + (rr & 7) * 16 + (kk % epc) * esz;
      if (PREC == LOGM_PREC_TF32X3) {
        const uint32_t hi = to_tf32(v);
        const uint32_t lo = to_tf32(v - __uint_as_float(hi));
        *reinterpret_cast<uint32_t*>(S.a + byte) = hi;
        *reinterpret_cast<uint32_t*>(S.a + a_slice + byte) = lo;
      } else {
        const __nv_bfloat16 s0 = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(s0);
        const __nv_bfloat16 s1 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 s2 = __float2bfloat16_rn(r1 - __bfloat162float(s1));
        *reinterpret_cast<__nv_bfloat16*>(S.a + byte) = s0;
        *reinterpret_cast<__nv_bfloat16*>(S.a + a_slice + byte) = s1;
        *reinterpret_cast<__nv_bfloat16*>(S.a + 2 * a_slice + byte) = s2;
      }
    }
    // B tile: K rows k0..k0+31, columns c0..c0+N-1, stored transposed (K-major)
    for (int e = tid; e < kTcK * N; e += kTcThreads) {
      const int kk = e / N, cc = e % N;
      const int gk = k0 + kk, gc = c0 + cc;
      float v = 0.0f;
      if (gk < n && gc < n) {
        const int64_t idx = (int64_t)gk * n + gc;
        for (int i = 0; i < cf.terms; ++i) v = fmaf(cf.g[i], P[i][idx], v);
      }
      const int byte = (cc >> 3) * sbo + (kk / epc) * 128 + (cc & 7) * 16 + (kk % epc) * esz;
      if (PREC == LOGM_PREC_TF32X3) {
        const uint32_t hi = to_tf32(v);
        const uint32_t lo = to_tf32(v - __uint_as_float(hi));
        *reinterpret_cast<uint32_t*>(S.b + byte) = hi;
        *reinterpret_cast<uint32_t*>(S.b + b_slice + byte) = lo;
      } else {
        const __nv_bfloat16 s0 = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(s0);
        const __nv_bfloat16 s1 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 s2 = __float2bfloat16_rn(r1 - __bfloat162float(s1));
        *reinterpret_cast<__nv_bfloat16*>(S.b + byte) = s0;
        *reinterpret_cast<__nv_bfloat16*>(S.b + b_slice + byte) = s1;
        *reinterpret_cast<__nv_bfloat16*>(S.b + 2 * b_slice + byte) = s2;
      }
    }
    // generic-proxy smem writes -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t a0 = smem_u32(S.a), b0 = smem_u32(S.b);
      for (int ks = 0; ks < kTcK / (32 / esz); ++ks) {  // one MMA covers 32 bytes of K
        const uint32_t ko = ks * 256;
        if (PREC == LOGM_PREC_TF32X3) {
          const uint64_t ah = sdesc(a0 + ko, 128, sbo), al = sdesc(a0 + a_slice + ko, 128, sbo);
          const uint64_t bh = sdesc(b0 + ko, 128, sbo), bl = sdesc(b0 + b_slice + ko, 128, sbo);
          mma_tf32(tmem, al, bh, id, (kc | ks) != 0);
          mma_tf32(tmem, ah, bl, id, 1);
          mma_tf32(tmem, ah, bh, id, 1);
        } else {
          uint64_t ad[3], bd[3];
          for (int t = 0; t < 3; ++t) {
            ad[t] = sdesc(a0 + t * a_slice + ko, 128, sbo);
            bd[t] = sdesc(b0 + t * b_slice + ko, 128, sbo);
          }
          mma_bf16(tmem, ad[2], bd[0], id, (kc | ks) != 0);
          mma_bf16(tmem, ad[1], bd[1], id, 1);
          mma_bf16(tmem, ad[0], bd[2], id, 1);
          mma_bf16(tmem, ad[1], bd[0], id, 1);
          mma_bf16(tmem, ad[0], bd[1], id, 1);
          mma_bf16(tmem, ad[0], bd[0], id, 1);
        }
      }
      mma_commit(mbar);
    }
    // wait until the MMAs that read this round's tiles have completed
    if (!mbar_wait(mbar, phase)) failed = 1;
    phase ^= 1;
    fence_after();
    if (__syncthreads_or(failed)) {
      failed = 1;
      break;
    }
  }

  if (!failed) {
    // epilogue: TMEM -> registers; warp w reads lanes 32 (w % 4).. of its column half
    const int sp = warp & 3, half = warp >> 2;
    const int row = r0 + sp * 32 + lane;
    const int cbeg = half * (N / 2), cend = cbeg + N / 2;  // N/2 is a multiple of 8
    const int last = is_last_product(k, p.j);
    const float scale = (last && p.s_dev) ? -ldexpf(1.0f, p.s_dev[b]) : 1.0f;
    float yv[6] = {0, 0, 0, 0, 0, 0};
    float ylast = 0.0f;
    if (last) {
      for (int i = 0; i <= p.j - 1 && i < 5; ++i) yv[i] = scheme_y(k, i);
      ylast = scheme_y(k, p.j);
    }
    float* outP = p.gbuf + ((int64_t)b * 5 + min(p.j, 4)) * nn_max;  // P_{j+2} slot (j <= 4)
    for (int cb = cbeg; cb < cend; cb += 8) {
      uint32_t r[8];
      const uint32_t ta = tmem + (static_cast<uint32_t>(sp * 32) << 16) + static_cast<uint32_t>(cb);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(ta));
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
            if (p.bal) v *= (float)(p.bal[(int64_t)b * p.n_max + row] / p.bal[(int64_t)b * p.n_max + gc]);
            if (p.out_dtype == 0)
              static_cast<double*>(p.L)[off + idx] = static_cast<double>(v);
            else
              static_cast<float*>(p.L)[off + idx] = v;
          }
        }
      }
    }
  } else {
    if (tid == 0 && p.err) atomicExch(p.err, 1);
    mbar_wait(mbar, phase ^ 1);  // bounded second wait for MMAs still in flight
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// Final step of matrices evaluated with k = 1 (no product after P_3):
// L = scale (X + X^2 / 2).
__global__ void k_graph_k1(GraphParams p) {
  const int b = blockIdx.y;
  int n;
  int64_t off;
  if (p.n_uniform > 0) {
    n = p.n_uniform;
    off = (int64_t)b * n * n;
  } else {
    n = p.n_dev[b];
    off = p.off_dev[b];
  }
  if (p.info_dev && (p.info_dev[b] == 1 || p.info_dev[b] == 4)) return;
  if (p.k_dev[b] != 1 || n < 1 || n > p.n_max) return;
  const int64_t nn_max = (int64_t)p.n_max * p.n_max;
  const float* P2 = p.gbuf + (int64_t)b * 5 * nn_max;
  const float* P3 = P2 + nn_max;
  const float scale = p.s_dev ? -ldexpf(1.0f, p.s_dev[b]) : 1.0f;
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
    float v = scale * fmaf(0.5f, P3[t], P2[t]);
    if (p.bal) v *= (float)(p.bal[(int64_t)b * p.n_max + t / n] / p.bal[(int64_t)b * p.n_max + t % n]);
    if (p.out_dtype == 0)
      static_cast<double*>(p.L)[off + t] = static_cast<double>(v);
    else
      static_cast<float*>(p.L)[off + t] = v;
  }
}

// logm_graph_eval in a split precision: X (and P_3 if given) -> FP32 slots 0, 1.
__global__ void k_graph_prep(GraphParams p, const void* X, const void* P3, int in_dtype) {
  const int b = blockIdx.y;
  int n;
  int64_t off;
  if (p.n_uniform > 0) {
    n = p.n_uniform;
    off = (int64_t)b * n * n;
  } else {
    n = p.n_dev[b];
    off = p.off_dev[b];
  }
  if (n < 1 || n > p.n_max) return;
  const int64_t nn_max = (int64_t)p.n_max * p.n_max;
  float* g2 = p.gbuf + (int64_t)b * 5 * nn_max;
  float* g3 = g2 + nn_max;
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
    g2[t] = in_dtype == 0 ? static_cast<float>(static_cast<const double*>(X)[off + t])
                          : static_cast<const float*>(X)[off + t];
    if (P3)
      g3[t] = in_dtype == 0 ? static_cast<float>(static_cast<const double*>(P3)[off + t])
                            : static_cast<const float*>(P3)[off + t];
  }
}

cudaError_t launch_graph_prep(const GraphParams& p, const void* X, const void* P3, int in_dtype, cudaStream_t st) {
  if (p.count <= 0) return cudaSuccess;
  k_graph_prep<<<dim3(64, p.count), 256, 0, st>>>(p, X, P3, in_dtype);
  return cudaGetLastError();
}

size_t graph_tc_smem_bytes() { return sizeof(TcSmem); }

cudaError_t launch_graph_k1(const GraphParams& p, cudaStream_t st) {
  if (p.count <= 0) return cudaSuccess;
  GraphParams q = p;
  q.j = 1;
  k_graph_k1<<<dim3(64, p.count), 256, 0, st>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_graph_tc(const GraphParams& p, cudaStream_t st) {
  if (p.count <= 0) return cudaSuccess;
  const int n_pad = ((p.n_max + 15) / 16) * 16;
  const int tiles = ((p.n_max + kTcM - 1) / kTcM) * ((n_pad + kTcN - 1) / kTcN);
  const size_t smem = sizeof(TcSmem);
  static DeviceOnce attr;
  cudaError_t e = attr.run([&] {
    cudaError_t r =
        cudaFuncSetAttribute(k_graph_tc<LOGM_PREC_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r != cudaSuccess) return r;
    return cudaFuncSetAttribute(k_graph_tc<LOGM_PREC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const dim3 grid(tiles, p.count);
  for (int j = 1; j <= 5; ++j) {
    GraphParams q = p;
    q.j = j;
    if (p.precision == LOGM_PREC_TF32X3)
      k_graph_tc<LOGM_PREC_TF32X3><<<grid, kTcThreads, smem, st>>>(q);
    else
      k_graph_tc<LOGM_PREC_BF16X3><<<grid, kTcThreads, smem, st>>>(q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (j == 1) {
      k_graph_k1<<<dim3(64, p.count), 256, 0, st>>>(q);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace lg
