// tc_ptx.cuh -- inline-PTX wrappers for the Blackwell tensor-core path:
// shared-memory matrix and instruction descriptors for tcgen05.mma, TMEM
// fences, mbarrier waits with an iteration limit, and TMA tile copies.
// Shared by the split-precision graph products (graph_tma.cu) and the
// tensor-core Gauss-Jordan updates of the whole-GPU kernel (tc_update.cuh).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lg {

constexpr long long kTmWaitLimit = 1ll << 24;  // polls of an mbarrier before a wait gives up

static __device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzle layout: start address, leading byte offset (unused for this
// layout: 16 B), stride byte offset 1024 B (8 rows of 128 B), descriptor
// version 1, layout type 2 (128-byte swizzle).
static __device__ __forceinline__ uint64_t tm_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// The same for the 32-byte swizzle layout (rows of 16 BF16 = 32 B, 8-row
// groups 256 B apart): layout type 6.
static __device__ __forceinline__ uint64_t tm_desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(256 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(6) << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format fmt (kind::tf32:
// 2 = TF32; kind::f16: 0 = F16, 1 = BF16), both K-major, M x N.
static __device__ __forceinline__ uint32_t tm_idesc(uint32_t fmt, int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= fmt << 7;
  d |= fmt << 10;
  d |= static_cast<uint32_t>(N >> 3) << 17;
  d |= static_cast<uint32_t>(M >> 4) << 24;
  return d;
}

static __device__ __forceinline__ void tm_mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

static __device__ __forceinline__ void tm_mma_f16(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

static __device__ __forceinline__ void tm_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

static __device__ __forceinline__ bool tm_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kTmWaitLimit; ++it) {
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

static __device__ __forceinline__ void tm_bar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

static __device__ __forceinline__ void tm_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

static __device__ __forceinline__ void tm_load2d(uint32_t dst, const CUtensorMap* map, uint32_t mbar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(x), "r"(y)
      : "memory");
}

static __device__ __forceinline__ void tm_load3d(uint32_t dst, const CUtensorMap* map, uint32_t mbar, int x, int y,
                                                 int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

static __device__ __forceinline__ void tm_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
static __device__ __forceinline__ void tm_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Eight consecutive 32-bit TMEM columns of this thread's lane (32x32b shape:
// warp w reads lanes 32 (w % 4) .. + 31).
static __device__ __forceinline__ void tm_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}
static __device__ __forceinline__ void tm_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace lg
