// BF16 products of the precision form on the tensor cores with TMA operand
// loads: C (M x N, FP32, row-major) = A (M x Kd) * B (N x Kd)^T, both operands
// K-major BF16 in global memory (A = the BF16 copy of A or of A^T, B = the
// BF16 transposed factor; the products R and P of Alg. 1).  Split forms: an operand
// X is given as two BF16 arrays, X_hi = bf16(X) and X_lo = bf16(X - X_hi),
// whose sum carries X to about 16 significant bits.  With A split each stage
// holds both A tiles and C = A_hi B^T + A_lo B^T (two MMAs per K step, twice
// the A bytes: those of FP32 A); with both split C = A_hi B_hi^T +
// A_lo B_hi^T + A_hi B_lo^T (three MMAs; the lo x lo term is below 2^-16 of
// the product).  All MMAs are BF16 x BF16 with FP32 accumulation.
//
// One CTA per 128 x 128 output tile.  Warp 0 (one lane) streams K slices of
// 64 elements of A and B into a 6-stage ring of shared memory with
// cp.async.bulk.tensor (128-byte swizzle, completion counted on the stage's
// "full" mbarrier); warp 1 (one lane) waits for a full stage, issues four
// tcgen05.mma (kind::f16, K = 16 each) into the FP32 accumulator in tensor
// memory and commits to the stage's "empty" mbarrier; warps 2-5 wait for the
// final commit and move the accumulator TMEM -> registers -> global memory.
// Out-of-range rows / K are zero-filled by the TMA unit.  Every wait is
// bounded (ST_TIMEOUT).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "devutil.cuh"
#include "internal.cuh"
#include "tcutil.cuh"

namespace plnmf {
namespace {

constexpr int TM = 128, TN = 128, TK = 64;        // tile; TK BF16 = 128 bytes
constexpr int A_STAGE = TM * 128, B_STAGE = TN * 128;
// Operand modes: 0 = A and B as given; 1 = A split; 2 = A and B split.
// Ring depth: 6 x 32 KB in flight (4: P 59.7 -> 6: 56.2 us at 8192^2, K = 256);
// the split forms' 48 KB / 64 KB stages fit 4 / 3.
template <int MODE>
struct Ring {
  static constexpr int kA = MODE >= 1 ? 2 : 1;          // A tiles per stage
  static constexpr int kB = MODE == 2 ? 2 : 1;          // B tiles per stage
  static constexpr int kStage = kA * A_STAGE + kB * B_STAGE;
  static constexpr int kDepth = MODE == 0 ? 6 : (MODE == 1 ? 4 : 3);
  static constexpr size_t kSmem = (size_t)kDepth * kStage + 1024;
};
constexpr int NSTAGE = 6;                          // barrier slots (>= every ring depth)
constexpr int TMA_THREADS = 192;

__device__ __forceinline__ unsigned long long desc_sw128(unsigned saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
  d |= (unsigned long long)(16u >> 4) << 16;
  d |= (unsigned long long)(1024u >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

__device__ __forceinline__ bool wait_bounded(unsigned bar, unsigned parity, int* status) {
  unsigned long long t0 = 0;
  unsigned polls = 0;
  while (!mbar_try_wait_cta(bar, parity)) {
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

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    tc_tma_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapAlo,
                       const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapBlo, float* C,
                       int64_t ldc, int M, int N, int Kd, int kps, int64_t split_stride, int* status) {
  constexpr int DEPTH = Ring<MODE>::kDepth;
  constexpr int STAGE = Ring<MODE>::kStage;
  constexpr int NA = Ring<MODE>::kA;
  extern __shared__ __align__(1024) char smem_raw[];
  __shared__ __align__(8) unsigned long long full[NSTAGE], empty[NSTAGE], done;
  __shared__ unsigned tmem_base;
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  // Split K: this CTA adds K slice [k0, k1) (kps a multiple of TK) into its
  // own partial output C + z * split_stride.
  const int k0 = blockIdx.z * kps, k1 = min(Kd, k0 + kps);
  const int nk = k1 > k0 ? (k1 - k0 + TK - 1) / TK : 0;
  C += (int64_t)blockIdx.z * split_stride;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    fence_mbar_init();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // Producer.
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % DEPTH;
      if (kb >= DEPTH) ok = wait_bounded(smem_u32(&empty[s]), ((kb / DEPTH) - 1) & 1, status);
      if (!ok) break;
      const unsigned a = smem_u32(smem + s * STAGE);
      const unsigned b = a + NA * A_STAGE;
      mbar_arrive_expect_tx(smem_u32(&full[s]), STAGE);
      tma_load_2d(a, &mapA, k0 + kb * TK, m0, smem_u32(&full[s]));
      if (MODE >= 1) tma_load_2d(a + A_STAGE, &mapAlo, k0 + kb * TK, m0, smem_u32(&full[s]));
      tma_load_2d(b, &mapB, k0 + kb * TK, n0, smem_u32(&full[s]));
      if (MODE == 2) tma_load_2d(b + B_STAGE, &mapBlo, k0 + kb * TK, n0, smem_u32(&full[s]));
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer.
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TN >> 3) << 17) | ((unsigned)(TM >> 4) << 24);
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % DEPTH;
      ok = wait_bounded(smem_u32(&full[s]), (kb / DEPTH) & 1, status);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a = smem_u32(smem + s * STAGE);
      const unsigned b = a + NA * A_STAGE;
      // Term h: (A_hi, B_hi), (A_lo, B_hi), (A_hi, B_lo) as the mode has them.
#pragma unroll
      for (int h = 0; h < MODE + 1; ++h) {
        const unsigned ah = a + (h == 1 ? A_STAGE : 0), bh = b + (h == 2 ? B_STAGE : 0);
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk) {
          const unsigned long long ad = desc_sw128(ah + kk * 32), bd = desc_sw128(bh + kk * 32);
          const unsigned acc = (kb > 0 || kk > 0 || h > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&done))
                 : "memory");
  } else if (warp >= 2) {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31.
    const int q = warp & 3;
    const bool got = nk > 0 && wait_bounded(smem_u32(&done), 0, status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = m0 + q * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 16) {
      unsigned r[16];
      const unsigned taddr = tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
          "%13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m >= M) continue;
      float* crow = C + (int64_t)m * ldc + n0 + c0;
      if (n0 + c0 + 16 <= N && (ldc & 3) == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const float4 v = make_float4(got ? __uint_as_float(r[j]) : 0.f, got ? __uint_as_float(r[j + 1]) : 0.f,
                                       got ? __uint_as_float(r[j + 2]) : 0.f, got ? __uint_as_float(r[j + 3]) : 0.f);
          *reinterpret_cast<float4*>(crow + j) = v;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + c0 + j < N) crow[j] = got ? __uint_as_float(r[j]) : 0.f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  if (__syncthreads_or(ok ? 0 : 1)) drain_grace();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D BF16 tensor map: `rows` rows of `cols` elements (row stride ld
// elements), box 64 x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// dst (cols x ldd, BF16) = transpose of src (rows x cols, FP32, row stride lds);
// with lo != nullptr also lo = bf16(src - dst) (the split form's low part).
__global__ void transpose_bf16_kernel(const float* __restrict__ src, int rows, int cols, int64_t lds,
                                      __nv_bfloat16* __restrict__ dst, int64_t ldd, __nv_bfloat16* __restrict__ lo) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(int64_t)r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ldd) {
      const float x = r < rows ? tile[threadIdx.x][i] : 0.f;
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      dst[(int64_t)c * ldd + r] = h;
      if (lo) lo[(int64_t)c * ldd + r] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
}

}  // namespace

bool tma_map_f32(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                 int box_rows) {
  auto enc = get_encode();
  if (!enc || ((ld * 4) & 15) || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor-map encoding reachable and the kernels' shared-memory opt-in done
// (once per process, outside any stream capture).
bool tma_available() {
  static bool ok = false;
  static std::once_flag once;
  std::call_once(once, [] {
    ok = get_encode() != nullptr &&
         cudaFuncSetAttribute(tc_tma_bf16_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Ring<0>::kSmem) == cudaSuccess &&
         cudaFuncSetAttribute(tc_tma_bf16_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Ring<1>::kSmem) == cudaSuccess &&
         cudaFuncSetAttribute(tc_tma_bf16_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Ring<2>::kSmem) == cudaSuccess;
  });
  return ok;
}

cudaError_t transpose_to_bf16(const float* src, int rows, int cols, int64_t lds, void* dst, int64_t ldd,
                              cudaStream_t s, void* lo) {
  dim3 grid((cols + 31) / 32, (int)((ldd + 31) / 32));
  if (grid.y > 65535 || ldd < rows) return cudaErrorInvalidValue;
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, lds, static_cast<__nv_bfloat16*>(dst), ldd,
                                                     static_cast<__nv_bfloat16*>(lo));
  return cudaGetLastError();
}

namespace {
// One launch of the mode the given low parts select (B_lo needs A_lo).
cudaError_t launch_tma(const CUtensorMap& ma, const CUtensorMap* malo, const CUtensorMap& mb, const CUtensorMap* mblo,
                       dim3 grid, float* C, int64_t ldc, int M, int N, int Kd, int kps, int64_t stride, int* d_status,
                       cudaStream_t s) {
  if (malo && mblo)
    tc_tma_bf16_kernel<2><<<grid, TMA_THREADS, Ring<2>::kSmem, s>>>(ma, *malo, mb, *mblo, C, ldc, M, N, Kd, kps,
                                                                    stride, d_status);
  else if (malo)
    tc_tma_bf16_kernel<1><<<grid, TMA_THREADS, Ring<1>::kSmem, s>>>(ma, *malo, mb, mb, C, ldc, M, N, Kd, kps, stride,
                                                                    d_status);
  else
    tc_tma_bf16_kernel<0><<<grid, TMA_THREADS, Ring<0>::kSmem, s>>>(ma, ma, mb, mb, C, ldc, M, N, Kd, kps, stride,
                                                                    d_status);
  return cudaGetLastError();
}
}  // namespace

cudaError_t tc_bf16_tma_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int M,
                             int N, int Kd, int* d_status, cudaStream_t s, const void* A_lo, const void* B_lo) {
  if (M <= 0 || N <= 0 || Kd <= 0) return cudaSuccess;
  if (B_lo && !A_lo) return cudaErrorInvalidValue;
  // TMA rules: 16-byte aligned bases and row strides (multiples of 8 BF16).
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) ||
      (reinterpret_cast<uintptr_t>(A_lo) & 15) || (reinterpret_cast<uintptr_t>(B_lo) & 15) || (lda & 7) || (ldb & 7))
    return cudaErrorInvalidValue;
  if (!tma_available()) return cudaErrorNotSupported;
  CUtensorMap ma, malo, mb, mblo;
  if (!make_map(&ma, A, M, Kd, lda, TM) || !make_map(&mb, B, N, Kd, ldb, TN)) return cudaErrorInvalidValue;
  if (A_lo && !make_map(&malo, A_lo, M, Kd, lda, TM)) return cudaErrorInvalidValue;
  if (B_lo && !make_map(&mblo, B_lo, N, Kd, ldb, TN)) return cudaErrorInvalidValue;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  return launch_tma(ma, A_lo ? &malo : nullptr, mb, B_lo ? &mblo : nullptr, grid, C, ldc, M, N, Kd, Kd, 0, d_status,
                    s);
}

cudaError_t tc_bf16_tma_gram_partials(const void* Xt, int64_t ldx, int Kp, int N, float* part, int splits,
                                      int* d_status, cudaStream_t s, const void* Xt_lo) {
  if (Kp <= 0 || N <= 0 || splits < 1) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(Xt) & 15) || (reinterpret_cast<uintptr_t>(Xt_lo) & 15) || (ldx & 7))
    return cudaErrorInvalidValue;
  if (!tma_available()) return cudaErrorNotSupported;
  CUtensorMap m, mlo;
  if (!make_map(&m, Xt, Kp, N, ldx, TM)) return cudaErrorInvalidValue;
  if (Xt_lo && !make_map(&mlo, Xt_lo, Kp, N, ldx, TM)) return cudaErrorInvalidValue;
  const int kps = ((N + splits - 1) / splits + TK - 1) / TK * TK;
  dim3 grid((Kp + TN - 1) / TN, (Kp + TM - 1) / TM, splits);
  // Split factor: X_hi X_hi^T + X_lo X_hi^T + X_hi X_lo^T.
  return launch_tma(m, Xt_lo ? &mlo : nullptr, m, Xt_lo ? &mlo : nullptr, grid, part, Kp, Kp, Kp, N, kps,
                    (int64_t)Kp * Kp, d_status, s);
}

int tma_gram_splits(int Kp, int N) {
  const int tiles = ((Kp + TN - 1) / TN) * ((Kp + TM - 1) / TM);
  int splits = std::max(1, 148 / tiles);
  splits = std::min(splits, std::max(1, (N + TK - 1) / TK));     // at least one K slice each
  return std::min(splits, 256);
}

}  // namespace plnmf
