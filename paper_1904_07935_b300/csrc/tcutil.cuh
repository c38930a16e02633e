// Tensor-core (tcgen05) and TMA helpers for the kernels that form the
// factor updates' off-tile sums on the tensor cores (hupdate_tc.cu): shared-
// memory matrix descriptors, the instruction descriptor, MMA issue and
// commit, tensor-memory allocation and loads, 2-D tensor copies, the TF32
// split and bounded mbarrier waits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "devutil.cuh"

namespace plnmf {
namespace tc {

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (rows of 128 bytes: 32 TF32 or 64 BF16 elements).
__device__ __forceinline__ unsigned long long desc_sw128(unsigned saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);          // start address
  d |= (unsigned long long)(16u >> 4) << 16;                    // leading byte offset (unused: swizzled K-major)
  d |= (unsigned long long)(1024u >> 4) << 32;                  // stride byte offset: next 8-row atom
  d |= 1ull << 46;                                              // descriptor version
  d |= 2ull << 61;                                              // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulation, K-major A and B, M x N; operand
// format 1 = BF16 (kind::f16), 2 = TF32 (kind::tf32).
__host__ __device__ constexpr unsigned idesc(int m, int n, unsigned fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long ad, unsigned long long bd, unsigned id,
                                         unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(id), "r"(accumulate)
      : "memory");
}

// Arrives on the mbarrier once every MMA issued before it by this thread has
// completed.
__device__ __forceinline__ void commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes made visible to the tensor cores (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Whole warp: allocate `cols` TMEM columns (a power of two >= 32); the base
// address is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned base, unsigned cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
// Sixteen consecutive 32-bit columns of this thread's TMEM lane (warp w reads
// lanes 32 (w % 4) .. + 31; taddr carries the lane base in its high half).
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 2-D tiled bulk tensor copy global -> shared (coordinates: x = inner
// element index, a multiple of 16 bytes; y = row), completion on `bar`.
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Nearest TF32 value (10 fraction bits) of a, as an FP32 pattern.
__device__ __forceinline__ float tf32_rn(float a) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
  return __uint_as_float(r);
}

// Byte offset of (row r, byte b of its 128-byte row) in a K-major tile with
// the 128-byte swizzle (16-byte unit u of row r stored at unit u ^ (r mod 8)).
__device__ __forceinline__ unsigned sw128_off(int r, int b) {
  return (unsigned)((r >> 3) * 1024 + (r & 7) * 128 + ((((b >> 4) ^ (r & 7)) << 4) | (b & 15)));
}

// Bounded wait for phase `parity` of a CTA-local mbarrier; false once the
// limit (ns) has passed.
__device__ __forceinline__ bool wait(unsigned bar, unsigned parity, unsigned long long limit) {
  unsigned long long t0 = 0;
  unsigned polls = 0;
  while (!mbar_try_wait_cta(bar, parity)) {
    if ((++polls & 63u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit) return false;
    }
  }
  return true;
}

}  // namespace tc

// FP32 2-D tensor map for TMA: `rows` rows of `cols` elements, row stride ld
// elements (ld * 4 a multiple of 16), box box_cols x box_rows (box_cols * 4 =
// 128 with the swizzle), 128-byte swizzle, zero fill outside.  False if the
// driver's encoder is unavailable or rejects the arguments.
bool tma_map_f32(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                 int box_rows);

}  // namespace plnmf
