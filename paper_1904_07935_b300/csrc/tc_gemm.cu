// Tensor-core GEMM on the 5th-generation tensor cores (tcgen05) for the dense
// contractions of the iteration (Alg. 1): the Gram matrices W^T W and H H^T,
// phase 1 / phase 3 of the regrouped W update (Eqs. 4, 6) and the dense
// products A H^T, A^T W.
//
// C (M x N) = op(A) (M x K) * B (K x N) with the GemmArgs epilogues of the
// SIMT family.  One CTA computes a 128 x BN tile (BN <= 256, a multiple of
// 16) with the FP32 accumulator in tensor memory (TMEM).  Operands are staged
// by all threads from global memory into shared memory in the canonical
// K-major, 128-byte-swizzled layout (8-row atoms of 128-byte rows, 16-byte
// chunk c of row r stored at chunk c ^ (r mod 8)); one thread issues the
// tcgen05.mma instructions and commits them to an mbarrier per stage, so the
// staging of stage s + 1 overlaps the MMAs of stage s.
//
// Precision:
//  * TC_TF32X3 (FP32 inputs): every operand is split as a = hi + lo with
//    hi = tf32(a) (round to nearest) and lo = tf32(a - hi); the tile product
//    is hi*hi + hi*lo + lo*hi, accumulated in FP32 (error ~ 2^-21 relative per
//    product instead of TF32's 2^-11).
//  * TC_BF16 (BF16 products): operands rounded to BF16 (A may already be
//    stored as BF16), FP32 accumulation.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace plnmf {
namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 256;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): K-major, 128-byte swizzle, 8-row
// atoms 1024 bytes apart.
__device__ __forceinline__ unsigned long long sw128_desc(unsigned saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);          // start address
  d |= (unsigned long long)(16u >> 4) << 16;                    // leading byte offset (unused here)
  d |= (unsigned long long)(1024u >> 4) << 32;                  // stride byte offset: next 8-row atom
  d |= 1ull << 46;                                              // descriptor version
  d |= 2ull << 61;                                              // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M x N.
__host__ __device__ constexpr unsigned make_idesc(int m, int n, unsigned ab_format) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((unsigned)(n >> 3) << 17) |
         ((unsigned)(m >> 4) << 24);
}
constexpr unsigned kFmtBF16 = 1;   // kind::f16 operand format
constexpr unsigned kFmtTF32 = 2;   // kind::tf32 operand format

__device__ __forceinline__ void mbar_init(unsigned a, unsigned c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(c) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait; returns false (and sets ST_TIMEOUT) if the phase never came.
__device__ bool mbar_wait(unsigned a, unsigned parity, int* status) {
  unsigned long long t0 = 0;
  unsigned polls = 0;
  while (!mbar_try(a, parity)) {
    if ((++polls & 63u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kWaitLimitNs) {
        atomicOr(status, ST_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

__device__ __forceinline__ void drain_grace_tc() {
  const unsigned long long t0 = global_ns();
  while (global_ns() - t0 < 2000000ull) {
  }
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

template <bool TF32>
__device__ __forceinline__ void tc_mma(unsigned tmem_d, unsigned long long ad, unsigned long long bd,
                                       unsigned idesc, unsigned accumulate) {
  if (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void tc_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ float tf32_rn(float a) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
  return __uint_as_float(r);
}

// Byte offset of element (row r, k) (4-byte elements, 32 per 128-byte row) or
// (row r, k) for 2-byte elements (64 per row) inside a swizzled K-major tile.
__device__ __forceinline__ unsigned sw128_off(int r, int byte_in_row) {
  const int chunk = byte_in_row >> 4;
  return (unsigned)((r >> 3) * 1024 + (r & 7) * 128 + (((chunk ^ (r & 7)) << 4) | (byte_in_row & 15)));
}

struct TcTile {
  // Source accessor: element (r, k) of the operand tile is
  // src[(row0 + r) * rs + (k0 + k) * ks], valid for row0 + r < rows and
  // k0 + k < kdim.
  const float* src;
  const __nv_bfloat16* src_bf16;
  int64_t rs, ks;
  int rows, kdim;
  int mask_mode;   // 1: phase-1 mask, keep (k, n) only for k > n (B operand, n = row index)
};

// Stage one 32-wide (TF32, 128 bytes) or 64-wide (BF16, 128 bytes) K slice of
// an operand tile with `nrows` rows.  hi/lo: destination tiles (lo unused for
// BF16).
template <bool TF32>
__device__ __forceinline__ void stage_operand(const TcTile& t, int row0, int k0, int nrows, char* hi, char* lo) {
  constexpr int KW = TF32 ? 32 : 64;                 // elements per 128-byte row
  const int total = nrows * KW;
  const bool k_contig = (t.ks == 1);
  for (int e = threadIdx.x; e < total; e += TC_THREADS) {
    int r, k;
    if (k_contig) { r = e / KW; k = e % KW; }       // consecutive threads walk along k
    else { k = e / nrows; r = e % nrows; }          // consecutive threads walk along rows
    const int gr = row0 + r, gk = k0 + k;
    float v = 0.f;
    const bool inb = gr < t.rows && gk < t.kdim && !(t.mask_mode == 1 && !(gk > gr));
    if (inb) {
      const int64_t idx = (int64_t)gr * t.rs + (int64_t)gk * t.ks;
      v = t.src_bf16 ? __bfloat162float(t.src_bf16[idx]) : __ldg(t.src + idx);
    }
    if (TF32) {
      const float h = tf32_rn(v);
      const float l = tf32_rn(v - h);
      const unsigned off = sw128_off(r, k * 4);
      *reinterpret_cast<float*>(hi + off) = h;
      *reinterpret_cast<float*>(lo + off) = l;
    } else {
      const unsigned off = sw128_off(r, k * 2);
      *reinterpret_cast<__nv_bfloat16*>(hi + off) = __float2bfloat16_rn(v);
    }
  }
}

struct TcParams {
  GemmArgs g;
  const __nv_bfloat16* a_bf16;   // optional BF16 copy of A (BF16 mode)
  int* status;
};

template <bool TF32, int BN>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(TcParams P) {
  constexpr int A_BYTES = TC_M * 128;
  constexpr int B_BYTES = BN * 128;
  constexpr int NPROD = TF32 ? 2 : 1;               // hi (and lo) copies per operand
  constexpr int STAGE_BYTES = NPROD * (A_BYTES + B_BYTES);
  constexpr int KSTAGE = TF32 ? 32 : 64;             // K elements per stage
  constexpr int KMMA = TF32 ? 8 : 16;                // K per instruction
  constexpr unsigned TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  extern __shared__ __align__(1024) char smem_raw[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ unsigned tmem_base_sh;

  const GemmArgs& g = P.g;
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * BN;
  const int z = blockIdx.z;
  int k_begin = 0, k_end = g.Kin;
  if (g.mode == GM_PARTIAL) {
    k_begin = z * g.k_chunk;
    k_end = min(g.Kin, k_begin + g.k_chunk);
  }
  if (g.mode == GM_PHASE1) k_begin = (n0 + 1) / KSTAGE * KSTAGE;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_sh)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_addr(&mbar[0]), 1);
    mbar_init(smem_addr(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_base_sh;

  // Operand accessors.  A: op(A)[m][k]; B (as the MMA's N x K operand): B[k][n].
  TcTile ta;
  ta.src = g.A;
  ta.src_bf16 = P.a_bf16;
  ta.rs = g.transA ? 1 : g.lda;
  ta.ks = g.transA ? g.lda : 1;
  ta.rows = g.M;
  ta.kdim = k_end;
  ta.mask_mode = 0;
  TcTile tb;
  tb.src = g.B;
  tb.src_bf16 = nullptr;
  tb.rs = 1;
  tb.ks = g.ldb;
  tb.rows = g.N;
  tb.kdim = k_end;
  tb.mask_mode = g.mode == GM_PHASE1 ? 1 : 0;

  const unsigned idesc = make_idesc(TC_M, BN, TF32 ? kFmtTF32 : kFmtBF16);
  const int nst = k_end > k_begin ? (k_end - k_begin + KSTAGE - 1) / KSTAGE : 0;
  bool ok = true;
  for (int s = 0; s < nst; ++s) {
    const int buf = s & 1;
    char* st = smem + buf * STAGE_BYTES;
    char* a_hi = st;
    char* b_hi = st + A_BYTES;
    char* a_lo = st + A_BYTES + B_BYTES;
    char* b_lo = a_lo + A_BYTES;
    if (s >= 2 && ok) ok = mbar_wait(smem_addr(&mbar[buf]), ((s - 2) >> 1) & 1, P.status);
    const int k0 = k_begin + s * KSTAGE;
    stage_operand<TF32>(ta, m0, k0, TC_M, a_hi, a_lo);
    stage_operand<TF32>(tb, n0, k0, BN, b_hi, b_lo);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < KSTAGE / KMMA; ++kk) {
        const unsigned koff = kk * KMMA * (TF32 ? 4 : 2);
        const unsigned long long ah = sw128_desc(smem_addr(a_hi) + koff);
        const unsigned long long bh = sw128_desc(smem_addr(b_hi) + koff);
        tc_mma<TF32>(tmem, ah, bh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
        if (TF32) {
          const unsigned long long al = sw128_desc(smem_addr(a_lo) + koff);
          const unsigned long long bl = sw128_desc(smem_addr(b_lo) + koff);
          tc_mma<TF32>(tmem, ah, bl, idesc, 1u);
          tc_mma<TF32>(tmem, al, bh, idesc, 1u);
        }
      }
      tc_commit(smem_addr(&mbar[buf]));
    }
  }
  // Wait for the last commit (it tracks every earlier MMA of this thread).
  if (nst > 0 && ok) ok = mbar_wait(smem_addr(&mbar[(nst - 1) & 1]), ((nst - 1) >> 1) & 1, P.status);
  tc_fence_after();

  // Epilogue: warps 0-3 read TMEM lanes 32w..32w+31 (rows of the tile).
  if (warp < 4) {
    const int m = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      unsigned r[16];
      const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
          "%13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + c0 + j;
        if (n >= g.N) continue;
        const float v = nst > 0 ? __uint_as_float(r[j]) : 0.f;
        switch (g.mode) {
          case GM_STORE:
            g.C[(int64_t)m * g.ldc + n] = v;
            break;
          case GM_PHASE1: {
            float base = g.E[(int64_t)m * g.lde + n];
            if (g.h_mode) base = fmaf(1.f - g.B[(int64_t)n * g.ldb + n], g.X[(int64_t)m * g.ldx + n], base);
            g.C[(int64_t)m * g.ldc + n] = base - v;
            break;
          }
          case GM_SUB:
            g.C[(int64_t)m * g.ldc + n] -= v;
            break;
          case GM_PARTIAL:
            g.C[(int64_t)z * g.part_stride + (int64_t)m * g.ldc + n] = v;
            break;
        }
      }
    }
  }
  tc_fence_before();
  // After a timed-out wait MMAs may still write TMEM: bounded grace period
  // before the allocation is released.
  if (__syncthreads_or(ok ? 0 : 1)) drain_grace_tc();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <bool TF32, int BN>
cudaError_t launch_tc(const TcParams& p, cudaStream_t s) {
  constexpr int NPROD = TF32 ? 2 : 1;
  const size_t smem = 2 * NPROD * (TC_M * 128 + BN * 128) + 1024;
  auto kern = tc_gemm_kernel<TF32, BN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((p.g.N + BN - 1) / BN, (p.g.M + TC_M - 1) / TC_M, p.g.mode == GM_PARTIAL ? p.g.n_chunks : 1);
  kern<<<grid, TC_THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

template <bool TF32>
cudaError_t dispatch_bn(const TcParams& p, int bn, cudaStream_t s) {
  switch (bn) {
    case 32: return launch_tc<TF32, 32>(p, s);
    case 64: return launch_tc<TF32, 64>(p, s);
    case 128: return launch_tc<TF32, 128>(p, s);
    case 160: return launch_tc<TF32, 160>(p, s);
    case 256: return launch_tc<TF32, 256>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int tc_pick_bn(int N) {
  if (N <= 32) return 32;
  if (N <= 64) return 64;
  if (N <= 128) return 128;
  if (N <= 160) return 160;
  return 256;
}

cudaError_t tc_gemm_run(const GemmArgs& g, TcPrecision prec, const void* a_bf16, int bn, int* d_status,
                        cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.upper_only) return cudaErrorInvalidValue;
  TcParams p;
  p.g = g;
  p.a_bf16 = static_cast<const __nv_bfloat16*>(a_bf16);
  p.status = d_status;
  if (bn == 0) bn = tc_pick_bn(g.N);
  return prec == TC_TF32X3 ? dispatch_bn<true>(p, bn, s) : dispatch_bn<false>(p, bn, s);
}

}  // namespace plnmf
