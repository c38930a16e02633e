// FP32 SIMT GEMM family used by the FP32 path: dense products A H^T and
// A^T W (Alg. 1 for dense A), the Gram matrices W^T W and H H^T (Alg. 1),
// phase 1 of the regrouped factor update (Eq. 4 plus the old
// half of Eq. 5, as one strictly-upper masked GEMM) and phase 3 (Eq. 6).
//
// 64 x 64 output tile per 256-thread CTA, 4 x 4 register micro-tile per
// thread, k staged through shared memory 16 at a time (double-buffered via
// registers).  FP32 multiply-add; FP32 accumulation, blocked and compensated
// (blocks of 64 terms added to running sums with TwoSum, as in the 128 x 128
// kernel below, the running sums here in registers).
#include <algorithm>
#include <vector>

#include "devutil.cuh"
#include "internal.cuh"

namespace plnmf {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ float load_a(const GemmArgs& g, int m, int k) {
  if (m >= g.M || k >= g.Kin) return 0.f;
  return g.transA ? __ldg(g.A + (int64_t)k * g.lda + m) : __ldg(g.A + (int64_t)m * g.lda + k);
}

__device__ __forceinline__ float load_b(const GemmArgs& g, int k, int n, int k_end) {
  if (k >= k_end || n >= g.N) return 0.f;
  if (g.mode == GM_PHASE1 && !(k > n)) return 0.f;   // strictly upper part only
  return g.transB ? __ldg(g.B + (int64_t)n * g.ldb + k) : __ldg(g.B + (int64_t)k * g.ldb + n);
}

__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
  __shared__ __align__(16) float As[2][BK][BM + 4];   // padded: conflict-light transposing stores
  __shared__ __align__(16) float Bs[2][BK][BN];

  int tm = blockIdx.y, tn = blockIdx.x;
  if (g.upper_only && tn < tm) return;
  const int m0 = tm * BM, n0 = tn * BN;
  const int z = blockIdx.z;
  int k_begin = 0, k_end = g.Kin;
  if (g.mode == GM_PARTIAL) {
    k_begin = z * g.k_chunk;
    k_end = min(g.Kin, k_begin + g.k_chunk);
  }
  if (g.mode == GM_PHASE1) {
    // B[k][n] with k <= n is masked: chunks entirely below n0 + 1 contribute nothing.
    k_begin = ((n0 + 1) / BK) * BK;
  }
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  // Loader mapping: 64 x 16 elements per operand, 4 per thread.
  // A: element (m = m0 + (tid & 63), k = kk + (tid >> 6) * 4 + i) for transA = 0 reads
  // along k; for transA = 1 the mapping is transposed so that reads run along m.
  float ra[4], rb[4];
  auto fetch = [&](int kk) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int e = tid + i * 256;                  // 0..1023
      int mm, kq;
      if (g.transA) { mm = e & 63; kq = e >> 6; } else { kq = e & 15; mm = e >> 4; }
      ra[i] = load_a(g, m0 + mm, kk + kq);
      int nn = e & 63, kb = e >> 6;
      rb[i] = load_b(g, kk + kb, n0 + nn, k_end);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int e = tid + i * 256;
      int mm, kq;
      if (g.transA) { mm = e & 63; kq = e >> 6; } else { kq = e & 15; mm = e >> 4; }
      As[buf][kq][mm] = ra[i];
      Bs[buf][e >> 6][e & 63] = rb[i];
    }
  };

  float acc[4][4], run[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = run[i][j] = 0.f;

  int buf = 0;
  if (k_begin < k_end) {
    fetch(k_begin);
    stash(0);
    __syncthreads();
    int steps = 0;
    for (int kk = k_begin; kk < k_end; kk += BK) {
      const bool more = kk + BK < k_end;
      if (more) fetch(kk + BK);
#pragma unroll
      for (int q = 0; q < BK; ++q) {
        const float4 a = *reinterpret_cast<const float4*>(&As[buf][q][ty * 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][q][tx * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float2 b01 = make_float2(b.x, b.y), b23 = make_float2(b.z, b.w);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 aa = make_float2(av[i], av[i]);
          fma_pair(acc[i][0], acc[i][1], aa, b01);
          fma_pair(acc[i][2], acc[i][3], aa, b23);
        }
      }
      if (++steps == 64 / BK) {                 // running sum += block; the error restarts the block
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) two_sum(run[i][j], acc[i][j], run[i][j], acc[i][j]);
        steps = 0;
      }
      if (more) {
        stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = run[i][j] + acc[i][j];

  // Epilogue.
  double r2 = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      const float v = acc[i][j];
      switch (g.mode) {
        case GM_STORE:
          g.C[(int64_t)m * g.ldc + n] = v;
          break;
        case GM_PHASE1: {
          const float e = g.E[(int64_t)m * g.lde + n];
          float base = e;
          if (g.h_mode) {
            const float cdiag = 1.f - g.B[(int64_t)n * g.ldb + n];
            base = fmaf(cdiag, g.X[(int64_t)m * g.ldx + n], e);
          }
          g.C[(int64_t)m * g.ldc + n] = base - v;
          break;
        }
        case GM_SUB:
          g.C[(int64_t)m * g.ldc + n] -= v;
          break;
        case GM_PARTIAL:
          g.C[(int64_t)z * g.part_stride + (int64_t)m * g.ldc + n] = v;
          break;
        case GM_RESID2: {
          const double d = (double)g.E[(int64_t)m * g.lde + n] - (double)v;
          r2 += d * d;
          break;
        }
      }
    }
  }
  if (g.mode == GM_RESID2) {
    __shared__ double red[256];
    red[threadIdx.x] = r2;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
      if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) g.dpart[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
  }
}

// Split-N Gram for 64 <= Kp <= 512: CTA (z, y) computes tile group y of the
// upper triangle of the Kp8 x Kp8 Gram of row chunk z (Kp8 = Kp rounded up
// to 8).  The Kp8
// indices form m = Kp8 / 8 groups of 8, group g = {4g .. 4g+3} together with
// {Kh + 4g .. Kh + 4g+3} (Kh = Kp8 / 2), so that consecutive groups are
// consecutive 16-byte words of a staged row (conflict-free loads).  Every
// pair of groups a <= b is one 8 x 8 register tile (m (m + 1) / 2 tiles),
// which covers every unordered index pair once (both orders for a = b); a
// value for (i, j) is stored at (min(i, j), max(i, j)) of the partial, the
// upper triangle that gram_reduce reads.  Two threads share a tile: rows of
// X are staged GR at a time in shared memory (double-buffered through
// registers) and thread half h multiplies rows [h GR/2, (h+1) GR/2) of each
// staged block; at the end half 1's tile goes through shared memory and half
// 0 adds it (fixed order).  The tiles are numbered row-major over the
// triangle and dealt in groups of tpg <= 253 (one group up to Kp = 176);
// every CTA of a chunk stages the same rows.
constexpr int GR = 16;                            // rows per staged block
constexpr int kGramFullMaxKp = kMaxK;             // up to m = 64: 2,080 tiles in 9 groups
constexpr int kTriGroupMax = 253;                 // tiles per CTA (506 threads)
constexpr int kGramFullMinKp = 64;                // m = 8: 36 tiles, 72 threads
__host__ __device__ constexpr int gram_tri_tiles(int Kp8) { return (Kp8 / 8) * (Kp8 / 8 + 1) / 2; }
constexpr int kTriStride = 256;                   // >= kTriGroupMax; compile-time offsets
__host__ __device__ constexpr int gram_tri_smem_floats(int Kp8) {
  return 2 * GR * Kp8 > 64 * kTriStride ? 2 * GR * Kp8 : 64 * kTriStride;
}
static_assert(kTriGroupMax <= kTriStride, "tile stride");
__global__ void __launch_bounds__(512) gram_tri_kernel(const float* __restrict__ X, int N, int Kp, int Kp8,
                                                       int chunk, int tpg, float* __restrict__ part,
                                                       const int* __restrict__ skip_count, int skip_need) {
  extern __shared__ __align__(16) float xs[];      // staging 2 x GR x Kp8; afterwards half 1's tiles
  // The partials are already there (formed in the same order by the W
  // update's workers): nothing to do.
  if (skip_count && *skip_count >= skip_need) return;
  const int m = Kp8 / 8, Kh = Kp8 / 2;
  const int nT = m * (m + 1) / 2;
  const int h = threadIdx.x >= tpg ? 1 : 0;
  const int ul = threadIdx.x - h * tpg;            // tile within the group
  const int ut = blockIdx.y * tpg + ul;            // tile within the triangle
  const bool act = ut < nT;                        // (the last group may be short)
  // Tile ut -> (ty, tx), ty <= tx, row-major over the upper triangle.
  int ty = 0, rem = act ? ut : 0;
  while (rem >= m - ty) {
    rem -= m - ty;
    ++ty;
  }
  const int tx = ty + rem;
  const int r0 = blockIdx.x * chunk, r1 = min(N, r0 + chunk);
  // acc[i][jj] holds columns 2 jj and 2 jj + 1 of tile row i (packed FP32
  // multiply-adds, each half rounded as a scalar fmaf).
  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  // Staging by 16-byte cp.async copies (L2 only; rows past the chunk and
  // columns past Kp zero-filled by the copy), the next block in flight while
  // the current one is multiplied.
  const int nt = blockDim.x;
  const int kq = Kp8 / 4;                          // 16-byte words per staged row
  const int total = GR * kq;
  auto stage = [&](int buf, int rb) {
    for (int e = threadIdx.x; e < total; e += nt) {
      const int r = e / kq, q = e % kq;
      const int row = rb + r;
      const bool ok = row < r1 && 4 * q < Kp;
      const float* src = ok ? X + (int64_t)row * Kp + 4 * q : X;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(xs + buf * GR * Kp8 + 4 * e)),
                   "l"(src), "r"(ok ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int buf = 0;
  stage(0, r0);
  for (int rb = r0; rb < r1; rb += GR) {
    const bool more = rb + GR < r1;
    if (more) {
      stage(buf ^ 1, rb + GR);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();                               // block rb landed for every thread
    const float* src = xs + buf * GR * Kp8 + h * (GR / 2) * Kp8;
#pragma unroll 2
    for (int r = 0; r < GR / 2; ++r) {
      const float* row = src + r * Kp8;
      const float4 a0 = *reinterpret_cast<const float4*>(row + 4 * ty);
      const float4 a1 = *reinterpret_cast<const float4*>(row + Kh + 4 * ty);
      const float4 b0 = *reinterpret_cast<const float4*>(row + 4 * tx);
      const float4 b1 = *reinterpret_cast<const float4*>(row + Kh + 4 * tx);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                            make_float2(b1.z, b1.w)};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 a = make_float2(av[i], av[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __ffma2_rn(a, bv[j], acc[i][j]);
      }
    }
    __syncthreads();                               // buf is free for the copies two blocks on
    buf ^= 1;
  }
  // Half 1 hands its tile to half 0 (entry-major with a fixed stride, so a
  // warp's accesses are consecutive words); the staging buffers are no longer
  // read.
  if (h == 1) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) xs[(i * 8 + j) * kTriStride + ul] = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
  }
  __syncthreads();
  if (h == 1 || !act) return;
  float* out = part + (int64_t)blockIdx.x * Kp * Kp;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int ri = i < 4 ? 4 * ty + i : Kh + 4 * ty + i - 4;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cj = j < 4 ? 4 * tx + j : Kh + 4 * tx + j - 4;
      const float v = ((j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x) + xs[(i * 8 + j) * kTriStride + ul];
      if (ri < Kp && cj < Kp) out[(int64_t)min(ri, cj) * Kp + max(ri, cj)] = v;
    }
    // One tile row at a time: keeps the compiler from hoisting all 64
    // shared-memory reads above the stores (register spills).
    asm volatile("" ::: "memory");
  }
}

// Large products (dense A H^T and A^T W): 128 x 128 output tile per
// 256-thread CTA, 8 x 8 register tile per thread (rows ty*4 + {0..3} and
// 64 + ty*4 + {0..3}, columns likewise with tx), k staged 8 at a time through
// shared memory (double-buffered via registers, one 16-byte global load per
// operand per thread and step).  Operands need 16-byte aligned bases and row
// strides that are multiples of 4 floats (checked by the caller).  Modes
// GM_STORE and GM_PARTIAL (upper_only: tiles below the diagonal skipped).
//
// Accumulation is blocked and compensated: the registers gather 64 terms
// (kFoldTiles k-steps of SBK), then each is added to its running sum with
// TwoSum; the running sums live in dynamic shared memory (64 floats per
// thread, laid out so that a warp's 16-byte accesses are conflict-free) and
// the exact rounding error of each addition stays in the register as the
// start of the next block.  Over a sum of L terms the error is then about
// one rounding of the result plus sqrt(64) roundings of a 64-term block,
// instead of about sqrt(L) roundings of the result (the dense factor updates
// cancel most of P and R, which magnifies the products' error).
constexpr int SB = 128, SBK = 8, SLD = SB + 4;
constexpr int kFoldTiles = 8;
constexpr int kSgemmThreads = 256;
constexpr size_t kSgemmDynSmem = sizeof(float4) * 16 * kSgemmThreads;   // 64 KB of running sums

// Elements (r, c .. c + 3) of a row-major matrix, zero outside rows < rmax,
// columns < cmax.
__device__ __forceinline__ float4 ldg4_guard(const float* __restrict__ base, int64_t ld, int r, int c, int rmax,
                                             int cmax) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r >= rmax) return v;
  const float* p = base + (int64_t)r * ld + c;
  if (c + 3 < cmax) return __ldg(reinterpret_cast<const float4*>(p));
  if (c < cmax) v.x = __ldg(p);
  if (c + 1 < cmax) v.y = __ldg(p + 1);
  if (c + 2 < cmax) v.z = __ldg(p + 2);
  return v;
}

__global__ void __launch_bounds__(kSgemmThreads, 2) sgemm128_kernel(GemmArgs g) {
  __shared__ __align__(16) float As[2][SBK][SLD];
  __shared__ __align__(16) float Bs[2][SBK][SLD];
  extern __shared__ float4 run_sum[];                         // [16][256]: this thread's at [q * 256 + tid]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (g.upper_only && blockIdx.x < blockIdx.y) return;        // Gram: tiles below the diagonal are not needed
  const int m0 = blockIdx.y * SB, n0 = blockIdx.x * SB;
  int k_begin = 0, k_end = g.Kin;
  if (g.mode == GM_PARTIAL) {
    k_begin = blockIdx.z * g.k_chunk;
    k_end = min(g.Kin, k_begin + g.k_chunk);
  }
  float4 ra, rb;
  auto fetch = [&](int kk) {
    if (!g.transA) ra = ldg4_guard(g.A, g.lda, m0 + (tid >> 1), kk + (tid & 1) * 4, g.M, k_end);
    else ra = ldg4_guard(g.A, g.lda, kk + (tid >> 5), m0 + (tid & 31) * 4, k_end, g.M);
    if (!g.transB) rb = ldg4_guard(g.B, g.ldb, kk + (tid >> 5), n0 + (tid & 31) * 4, k_end, g.N);
    else rb = ldg4_guard(g.B, g.ldb, n0 + (tid >> 1), kk + (tid & 1) * 4, g.N, k_end);
  };
  auto stash = [&](int buf) {
    if (!g.transA) {
      const int m = tid >> 1, kq = (tid & 1) * 4;
      As[buf][kq][m] = ra.x;
      As[buf][kq + 1][m] = ra.y;
      As[buf][kq + 2][m] = ra.z;
      As[buf][kq + 3][m] = ra.w;
    } else {
      *reinterpret_cast<float4*>(&As[buf][tid >> 5][(tid & 31) * 4]) = ra;
    }
    if (!g.transB) {
      *reinterpret_cast<float4*>(&Bs[buf][tid >> 5][(tid & 31) * 4]) = rb;
    } else {
      const int n = tid >> 1, kq = (tid & 1) * 4;
      Bs[buf][kq][n] = rb.x;
      Bs[buf][kq + 1][n] = rb.y;
      Bs[buf][kq + 2][n] = rb.z;
      Bs[buf][kq + 3][n] = rb.w;
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) run_sum[q * kSgemmThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  // Running sum += block (TwoSum); the rounding error restarts the block.
  auto fold = [&]() {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      float4 r = run_sum[q * kSgemmThreads + tid];
      float* a = &acc[q >> 1][4 * (q & 1)];
      two_sum(r.x, a[0], r.x, a[0]);
      two_sum(r.y, a[1], r.y, a[1]);
      two_sum(r.z, a[2], r.z, a[2]);
      two_sum(r.w, a[3], r.w, a[3]);
      run_sum[q * kSgemmThreads + tid] = r;
    }
  };
  int buf = 0;
  if (k_begin < k_end) {
    fetch(k_begin);
    stash(0);
    __syncthreads();
    int steps = 0;
    for (int kk = k_begin; kk < k_end; kk += SBK) {
      const bool more = kk + SBK < k_end;
      if (more) fetch(kk + SBK);
#pragma unroll
      for (int q = 0; q < SBK; ++q) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][q][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][q][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][q][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][q][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                              make_float2(b1.z, b1.w)};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 aa = make_float2(av[i], av[i]);
#pragma unroll
          for (int j = 0; j < 4; ++j) fma_pair(acc[i][2 * j], acc[i][2 * j + 1], aa, bv[j]);
        }
      }
      if (++steps == kFoldTiles) {
        fold();
        steps = 0;
      }
      if (more) {
        stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
  float* C = g.C + (g.mode == GM_PARTIAL ? (int64_t)blockIdx.z * g.part_stride : 0);
  const bool vec = (g.ldc & 3) == 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= g.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + h * 64 + tx * 4;
      const float4 r = run_sum[(2 * i + h) * kSgemmThreads + tid];
      const float v[4] = {r.x + acc[i][4 * h], r.y + acc[i][4 * h + 1], r.z + acc[i][4 * h + 2],
                          r.w + acc[i][4 * h + 3]};
      float* dst = C + (int64_t)m * g.ldc + n;
      if (vec && n + 3 < g.N) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (n + j < g.N) dst[j] = v[j];
      }
    }
  }
}

// The 128 x 128 kernel applies: plain or partial products, operands 16-byte
// aligned with row strides that are multiples of 4 floats, wide enough.
bool use_sgemm128(const GemmArgs& a) {
  if (a.mode != GM_STORE && a.mode != GM_PARTIAL) return false;
  if (a.M < 64 || a.N < 96 || a.Kin < 64) return false;
  if ((a.lda & 3) || (a.ldb & 3)) return false;
  if ((reinterpret_cast<uintptr_t>(a.A) & 15) || (reinterpret_cast<uintptr_t>(a.B) & 15)) return false;
  return true;
}

// S[i][j] = sum_z part[z][i][j] for i <= j, mirrored.  Compensated FP32
// summation (a TwoSum cascade: the running sum plus the sum of its exact
// rounding errors), which is as accurate as summing in twice the working
// precision and rounding once, on the FP32 pipes (B300's FP64 rate is a
// small fraction of its FP32 rate).  Coalesced loads and one memory latency:
// a block covers 32 consecutive entries x 8 chunk lanes (a warp = 32 entries
// of one chunk lane); chunk lane c adds chunks c, c + 8, ... (all its loads
// issued before the first add), then the lanes' (sum, error) pairs are added
// for c = 0..7 through shared memory.  Fixed order, so the result does not
// depend on scheduling.
constexpr int kReduceLanes = 8, kReducePer = 32;     // n_chunks <= 256
__global__ void __launch_bounds__(256) gram_reduce32_kernel(const float* __restrict__ part, int n_chunks, int Kp,
                                                            int K, float* __restrict__ S) {
  __shared__ float sh_s[kReduceLanes][33], sh_e[kReduceLanes][33];
  const int ej = threadIdx.x & 31, cl = threadIdx.x >> 5;
  const int entry = blockIdx.x * 32 + ej;
  const int i = entry / Kp, j = entry % Kp;
  const bool inside = entry < Kp * Kp;
  const bool need = inside && i < K && j < K && j >= i;
  float s = 0.f, c = 0.f;
  if (need) {
    const size_t stride = (size_t)Kp * Kp;
    const float* src = part + (size_t)i * Kp + j;
    float v[kReducePer];
#pragma unroll
    for (int k = 0; k < kReducePer; ++k) {
      const int z = cl + kReduceLanes * k;
      v[k] = z < n_chunks ? src[z * stride] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kReducePer; ++k) {
      if (cl + kReduceLanes * k >= n_chunks) break;
      float e;
      two_sum(s, v[k], s, e);
      c += e;
    }
  }
  sh_s[cl][ej] = s;
  sh_e[cl][ej] = c;
  __syncthreads();
  if (cl != 0 || !inside) return;
  if (i >= K || j >= K) {
    S[(int64_t)i * Kp + j] = 0.f;
    return;
  }
  if (j < i) return;
  float t = 0.f, ct = 0.f;
#pragma unroll
  for (int q = 0; q < kReduceLanes; ++q) {
    float e;
    two_sum(t, sh_s[q][ej], t, e);
    ct += e + sh_e[q][ej];
  }
  const float f = t + ct;
  S[(int64_t)i * Kp + j] = f;
  S[(int64_t)j * Kp + i] = f;
}

// S[i][j] = sum_z part[z][i][j] (FP64, z ascending) for i <= j, mirrored.
__global__ void gram_reduce_kernel(const float* __restrict__ part, int n_chunks, int Kp, int K,
                                   float* __restrict__ S) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Kp) return;
  if (i >= K || j >= K) {
    S[(int64_t)i * Kp + j] = 0.f;
    return;
  }
  if (j < i) return;
  double s = 0.0;
  const size_t stride = (size_t)Kp * Kp;
  for (int z = 0; z < n_chunks; ++z) s += (double)part[z * stride + (size_t)i * Kp + j];
  const float f = (float)s;
  S[(int64_t)i * Kp + j] = f;
  S[(int64_t)j * Kp + i] = f;
}

}  // namespace

cudaError_t gemm_run(const GemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (use_sgemm128(a)) {
    static const cudaError_t attr = cudaFuncSetAttribute(sgemm128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)kSgemmDynSmem);
    if (attr != cudaSuccess) return attr;
    dim3 grid((a.N + SB - 1) / SB, (a.M + SB - 1) / SB, a.mode == GM_PARTIAL ? a.n_chunks : 1);
    sgemm128_kernel<<<grid, kSgemmThreads, kSgemmDynSmem, s>>>(a);
    return cudaGetLastError();
  }
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, a.mode == GM_PARTIAL ? a.n_chunks : 1);
  gemm_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// C (M x N, row stride ldc) = sum over z of part[z] (M x N contiguous),
// compensated FP32 (TwoSum cascade) in z order.
__global__ void partial_sum_kernel(const float* __restrict__ part, int n_chunks, int M, int N,
                                   float* __restrict__ C, int64_t ldc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  const int64_t stride = (int64_t)M * N;
  float s = 0.f, c = 0.f;
  for (int z = 0; z < n_chunks; ++z) {
    float err;
    two_sum(s, part[z * stride + e], s, err);
    c += err;
  }
  const int64_t m = e / N, n = e - m * N;
  C[m * ldc + n] = s + c;
}

int splitk_chunks(int M, int N, int Kin) {
  // Tile grid of the kernel gemm_run will pick for a plain product.
  const int tb = (M >= 64 && N >= 96 && Kin >= 64) ? SB : BM;
  const int tiles = ((N + tb - 1) / tb) * ((M + tb - 1) / tb);
  if (tiles >= 296) return 1;
  const int want = (296 + tiles - 1) / tiles;                 // about two CTAs per SM
  const int most = std::max(1, Kin / (4 * BK));              // at least four K steps each
  return std::max(1, std::min(std::min(want, most), 64));
}

cudaError_t gemm_run_split(GemmArgs a, float* part, int n_chunks, cudaStream_t s) {
  if (n_chunks <= 1 || !part || a.mode != GM_STORE) return gemm_run(a, s);
  float* C = a.C;
  const int64_t ldc = a.ldc;
  a.mode = GM_PARTIAL;
  a.k_chunk = ((a.Kin + n_chunks - 1) / n_chunks + BK - 1) / BK * BK;        // a multiple of SBK too
  a.n_chunks = (a.Kin + a.k_chunk - 1) / a.k_chunk;
  a.C = part;
  a.ldc = a.N;
  a.part_stride = (int64_t)a.M * a.N;
  cudaError_t e = gemm_run(a, s);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)a.M * a.N;
  partial_sum_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, a.n_chunks, a.M, a.N, C, ldc);
  return cudaGetLastError();
}

int64_t resid2_partials(int V, int D) { return (int64_t)((D + BN - 1) / BN) * ((V + BM - 1) / BM); }

cudaError_t resid2_dense(const float* A, int64_t lda, const float* W, const float* Ht, int V, int D, int K, int Kp,
                         double* dpart, double* out, cudaStream_t s) {
  GemmArgs a;
  a.M = V; a.N = D; a.Kin = K;
  a.A = W; a.lda = Kp; a.transA = 0;
  a.B = Ht; a.ldb = Kp; a.transB = 1;
  a.E = A; a.lde = lda;
  a.mode = GM_RESID2;
  a.dpart = dpart;
  cudaError_t e = gemm_run(a, s);
  if (e != cudaSuccess) return e;
  const int64_t n = resid2_partials(V, D);
  std::vector<double> h((size_t)n);
  if ((e = cudaMemcpyAsync(h.data(), dpart, sizeof(double) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  double t = 0.0;
  for (double v : h) t += v;
  *out = t;
  return cudaSuccess;
}

cudaError_t gram_setup(GramWork& g, int N, int Kp) {
  g.N = N;
  g.Kp = Kp;
  if (Kp >= kGramFullMinKp && Kp <= kGramFullMaxKp) {
    // gram_tri_kernel: the triangle's tiles in groups of at most
    // kTriGroupMax, and row chunks (of at least GR rows) such that chunks x
    // groups is about one CTA per SM.
    const int nT = gram_tri_tiles((Kp + 7) / 8 * 8);
    g.groups = (nT + kTriGroupMax - 1) / kTriGroupMax;
    g.tpg = (nT + g.groups - 1) / g.groups;
    const int want = std::max(1, 148 / g.groups);
    const int chunk = std::max(GR, (N + want - 1) / want);
    g.chunk = chunk;
    g.n_chunks = (N + chunk - 1) / chunk;
    return cudaMalloc(&g.d_part, sizeof(float) * (size_t)g.n_chunks * Kp * Kp);
  }
  // Enough chunks to cover about two waves of the 148 SMs (chunks of at
  // least 2 BK rows; at most 256 chunks, the compensated reduction's limit).
  // Upper-triangle tiles: 128 x 128 for Kp >= 96 (sgemm128_kernel), else 64 x 64.
  const int tw = Kp >= 96 ? 128 : 64;
  const int tiles = ((Kp + tw - 1) / tw) * ((Kp + tw - 1) / tw + 1) / 2;
  int want = std::max(1, (296 + tiles - 1) / tiles);
  int chunk = (N + want - 1) / want;
  chunk = std::max(2 * BK, ((chunk + BK - 1) / BK) * BK);
  chunk = std::max(chunk, ((N + 255) / 256 + BK - 1) / BK * BK);
  g.chunk = chunk;
  g.n_chunks = (N + chunk - 1) / chunk;
  return cudaMalloc(&g.d_part, sizeof(float) * (size_t)g.n_chunks * Kp * Kp);
}

cudaError_t gram_setup_tc(GramWork& g, int N, int Kp) {
  g.N = N;
  g.Kp = Kp;
  // 128-row M tiles; enough 32-row-aligned chunks of N for about one wave.
  const int mtiles = (Kp + 127) / 128;
  const int want = std::max(1, 148 / mtiles);
  int chunk = (N + want - 1) / want;
  chunk = std::max(64, (chunk + 31) / 32 * 32);
  g.chunk = chunk;
  g.n_chunks = (N + chunk - 1) / chunk;
  return cudaMalloc(&g.d_part, sizeof(float) * (size_t)g.n_chunks * Kp * Kp);
}

// Sum of n_chunks partial Grams (Kp x Kp each) into S, FP64, fixed order.
cudaError_t gram_reduce(const float* part, int n_chunks, int Kp, int K, float* S, cudaStream_t s) {
  if (n_chunks <= kReduceLanes * kReducePer) {
    gram_reduce32_kernel<<<(Kp * Kp + 31) / 32, 256, 0, s>>>(part, n_chunks, Kp, K, S);
  } else {
    dim3 grid((Kp + 127) / 128, Kp);
    gram_reduce_kernel<<<grid, 128, 0, s>>>(part, n_chunks, Kp, K, S);
  }
  return cudaGetLastError();
}

cudaError_t gram_run_tc(const GramWork& g, const float* X, float* S, int K, int* d_status, cudaStream_t s,
                        bool bf16) {
  GemmArgs a;
  a.M = g.Kp;
  a.N = g.Kp;
  a.Kin = g.N;
  a.A = X;
  a.lda = g.Kp;
  a.transA = 1;
  a.B = X;
  a.ldb = g.Kp;
  a.C = g.d_part;
  a.ldc = g.Kp;
  a.mode = GM_PARTIAL;
  a.k_chunk = g.chunk;
  a.part_stride = (int64_t)g.Kp * g.Kp;
  a.n_chunks = g.n_chunks;
  cudaError_t err = tc_gemm_run(a, bf16 ? TC_BF16 : TC_TF32X3, nullptr, 0, d_status, s);
  if (err != cudaSuccess) return err;
  return gram_reduce(g.d_part, g.n_chunks, g.Kp, K, S, s);
}

cudaError_t gram_run_scratch(const float* X, int N, int K, int64_t ldx, float* part, int n_chunks, int chunk,
                             float* S, cudaStream_t s) {
  GemmArgs a;
  a.M = K;
  a.N = K;
  a.Kin = N;
  a.A = X;
  a.lda = ldx;
  a.transA = 1;
  a.B = X;
  a.ldb = ldx;
  a.C = part;
  a.ldc = K;
  a.mode = GM_PARTIAL;
  a.k_chunk = chunk;
  a.part_stride = (int64_t)K * K;
  a.n_chunks = n_chunks;
  a.upper_only = 1;
  cudaError_t err = gemm_run(a, s);
  if (err != cudaSuccess) return err;
  return gram_reduce(part, n_chunks, K, K, S, s);
}

void gram_rechunk(GramWork& g, int chunk, int n_chunks) {
  g.chunk = chunk;
  g.n_chunks = n_chunks;
  if (!(g.Kp >= kGramFullMinKp && g.Kp <= kGramFullMaxKp)) return;
  // Tile groups so that chunks x groups covers the SMs about twice (the
  // order of each entry's sum does not depend on the grouping).
  const int nT = gram_tri_tiles((g.Kp + 7) / 8 * 8);
  int groups = std::max((nT + kTriGroupMax - 1) / kTriGroupMax, (2 * 148 + n_chunks - 1) / std::max(1, n_chunks));
  groups = std::min(groups, std::max(1, nT / 32));
  g.groups = groups;
  g.tpg = (nT + groups - 1) / groups;
}

bool gram_tri_single_group(const GramWork& g) {
  return g.Kp >= kGramFullMinKp && g.Kp <= kGramFullMaxKp && g.groups == 1;
}

void gram_free(GramWork& g) {
  cudaFree(g.d_part);
  g.d_part = nullptr;
}

cudaError_t gram_run(const GramWork& g, const float* X, float* S, int K, cudaStream_t s, const int* skip_count,
                     int skip_need) {
  if (g.Kp >= kGramFullMinKp && g.Kp <= kGramFullMaxKp) {
    const int Kp8 = (g.Kp + 7) / 8 * 8;
    const int threads = 2 * g.tpg;
    const size_t smem = sizeof(float) * gram_tri_smem_floats(Kp8);
    static const cudaError_t attr = cudaFuncSetAttribute(
        gram_tri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)(sizeof(float) * gram_tri_smem_floats((kGramFullMaxKp + 7) / 8 * 8)));
    if (attr != cudaSuccess) return attr;
    gram_tri_kernel<<<dim3(g.n_chunks, g.groups), threads, smem, s>>>(X, g.N, g.Kp, Kp8, g.chunk, g.tpg, g.d_part,
                                                                     skip_count, skip_need);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return gram_reduce(g.d_part, g.n_chunks, g.Kp, K, S, s);
  }
  if (skip_count) return cudaErrorInvalidValue;      // partials of the W update's workers: gram_tri_kernel's order only
  GemmArgs a;
  a.M = g.Kp;
  a.N = g.Kp;
  a.Kin = g.N;
  a.A = X;
  a.lda = g.Kp;
  a.transA = 1;
  a.B = X;
  a.ldb = g.Kp;
  a.C = g.d_part;
  a.ldc = g.Kp;
  a.mode = GM_PARTIAL;
  a.k_chunk = g.chunk;
  a.part_stride = (int64_t)g.Kp * g.Kp;
  a.n_chunks = g.n_chunks;
  a.upper_only = 1;
  cudaError_t err = gemm_run(a, s);
  if (err != cudaSuccess) return err;
  return gram_reduce(g.d_part, g.n_chunks, g.Kp, K, S, s);
}

}  // namespace plnmf
