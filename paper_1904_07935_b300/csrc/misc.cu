// Initialisation, column normalisation and FP64 reductions.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace plnmf {
namespace {

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output i (0-based) of the
// generator seeded with s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).
__device__ __forceinline__ unsigned long long splitmix_at(unsigned long long seed,
                                                          unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// dst[r * ld + c] = U[0,1) draw number r * sr + c * sc for c < cols; 0 for the
// padding columns cols <= c < ld.
__global__ void fill_uniform_kernel(float* dst, int rows, int cols, int ld, long long sr, long long sc,
                                    unsigned long long seed) {
  const long long n = (long long)rows * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    float v = 0.f;
    if (c < cols) {
      const unsigned long long x = splitmix_at(seed, (unsigned long long)(r * sr + c * sc));
      v = (float)(x >> 40) * (1.0f / 16777216.0f);
    }
    dst[e] = v;
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide FP64 sum in a fixed pattern; result valid in thread 0.
template <int NT>
__device__ double block_sum_d(double v) {
  __shared__ double ws[NT / 32];
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < NT / 32 ? ws[threadIdx.x] : 0.0;
    t = warp_sum_d(t);
  }
  __syncthreads();
  return t;
}

// One block per column: norm in FP64, then X[:, k] /= norm (rounded to FP32).
__global__ void normalize_columns_kernel(float* X, int N, int K, int ld) {
  const int k = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const double v = X[(int64_t)r * ld + k];
    s += v * v;
  }
  __shared__ float col_norm;
  const double t = block_sum_d<256>(s);
  if (threadIdx.x == 0) col_norm = (float)sqrt(t);
  __syncthreads();
  const float nrm = col_norm;
  for (int r = threadIdx.x; r < N; r += blockDim.x) X[(int64_t)r * ld + k] /= nrm;
}

constexpr int kObjThreads = 256;
constexpr int kSqBlocks = 64;          // blocks of the <S, Q> partials (partial[n_wp .. n_wp + 64))

// Error-free transformations (Knuth TwoSum; TwoProduct through fma) and the
// compensated dot product Dot2 of Ogita, Rump & Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26(6), 2005: the result is as accurate as if
// computed in twice the working precision, without FP64 arithmetic.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

struct Dot2 {
  float p = 0.f, c = 0.f;     // running sum and accumulated error terms
  __device__ __forceinline__ void add(float a, float b) {
    const float h = a * b;
    const float r = fmaf(a, b, -h);       // exact: a * b = h + r
    float s, q;
    two_sum(p, h, s, q);
    p = s;
    c += q + r;
  }
  __device__ __forceinline__ double value() const { return (double)p + (double)c; }
};

// partial[b] = <a, b> over this block's grid-stride share of [0, n); n is a
// multiple of 4 and the arrays 16-byte aligned (16-byte loads, two in flight).
__global__ void dot_partial_kernel(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                   double* __restrict__ partial) {
  Dot2 acc;
  const long long step = (long long)gridDim.x * blockDim.x;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const float4* x4 = reinterpret_cast<const float4*>(a);
  const float4* y4 = reinterpret_cast<const float4*>(b);
#pragma unroll 2
  for (long long i = i0; i < n / 4; i += step) {
    const float4 u = __ldg(x4 + i), v = __ldg(y4 + i);
    acc.add(u.x, v.x);
    acc.add(u.y, v.y);
    acc.add(u.z, v.z);
    acc.add(u.w, v.w);
  }
  const double t = block_sum_d<kObjThreads>(acc.value());
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// frob2 = normA2 - 2 sum(partial[0..n_wp)) + sum(partial[n_wp..n_wp + n_sq))
// (<W, P> and <S, Q> partials of dot_partial_kernel, added in a fixed order);
// appended to the history ring.
__global__ void objective_final_kernel(const double* __restrict__ partial, int n_wp, int n_sq, double normA2,
                                       double* __restrict__ hist, unsigned* counter, int hist_cap,
                                       double* __restrict__ last) {
  double wp = 0.0, sq = 0.0;
  for (int i = threadIdx.x; i < n_wp; i += blockDim.x) wp += partial[i];
  for (int i = threadIdx.x; i < n_sq; i += blockDim.x) sq += partial[n_wp + i];
  wp = block_sum_d<kObjThreads>(wp);
  sq = block_sum_d<kObjThreads>(sq);
  if (threadIdx.x == 0) {
    const unsigned it = *counter;
    const double f = normA2 - 2.0 * wp + sq;
    hist[it % hist_cap] = f;
    *counter = it + 1;
    if (last) *last = f;
  }
}

// out[block] = this block's share of the sum of squares of a dense matrix;
// *bad |= 1 if any entry is negative or not finite (Sec. 1: A is non-negative).
__global__ void sumsq_dense_kernel(const float* __restrict__ A, long long rows, long long cols, long long ld,
                                   double* __restrict__ out, int* __restrict__ bad) {
  double s = 0.0;
  int b = 0;
  const long long n = rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    const float v = A[r * ld + c];
    if (!(v >= 0.f) || !(v < INFINITY)) b = 1;
    s += (double)v * (double)v;
  }
  const double t = block_sum_d<256>(s);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
  if (b) atomicOr(bad, 1);
}

// dst[c][r] = src[r][c] for r < rows, c < cols (32 x 32 tiles through shared memory).
__global__ void transpose_kernel(const float* __restrict__ src, int rows, int cols, int lds,
                                 float* __restrict__ dst, int ldd) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = src[(int64_t)r * lds + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[(int64_t)c * ldd + r] = tile[threadIdx.x][i];
  }
}

// dst = bf16(src) (round to nearest even); with lo != nullptr also
// lo = bf16(src - dst), the split form's low part.
__global__ void convert_bf16_kernel(const float* __restrict__ src, long long rows, long long cols, long long lds,
                                    __nv_bfloat16* __restrict__ dst, long long ldd, __nv_bfloat16* __restrict__ lo) {
  const long long n = rows * ldd;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ldd, c = e - r * ldd;
    const float x = c < cols ? src[r * lds + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    dst[e] = h;
    if (lo) lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

}  // namespace

cudaError_t convert_bf16(const float* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                         cudaStream_t s, void* lo) {
  convert_bf16_kernel<<<1184, 256, 0, s>>>(src, rows, cols, lds, static_cast<__nv_bfloat16*>(dst), ldd,
                                           static_cast<__nv_bfloat16*>(lo));
  return cudaGetLastError();
}

cudaError_t transpose_f32(const float* src, int rows, int cols, int lds, float* dst, int ldd, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, lds, dst, ldd);
  return cudaGetLastError();
}

cudaError_t fill_uniform_splitmix(float* dst, int rows, int cols, int ld, uint64_t seed, cudaStream_t s) {
  // Not transposed: element (r, c) is draw r * cols + c.
  fill_uniform_kernel<<<592, 256, 0, s>>>(dst, rows, cols, ld, cols, 1, seed);
  return cudaGetLastError();
}

cudaError_t fill_uniform_splitmix_t(float* dst, int rows, int cols, int ld, uint64_t seed, cudaStream_t s) {
  // Transposed storage of a cols x rows matrix: element (r, c) is draw c * rows + r.
  fill_uniform_kernel<<<592, 256, 0, s>>>(dst, rows, cols, ld, 1, rows, seed);
  return cudaGetLastError();
}

cudaError_t normalize_columns(float* X, int N, int K, int ld, cudaStream_t s) {
  normalize_columns_kernel<<<K, 256, 0, s>>>(X, N, K, ld);
  return cudaGetLastError();
}

cudaError_t objective_wp(const float* W, const float* P, int V, int Kp, double* partial, int n_partial,
                         cudaStream_t s) {
  if (Kp & 3) return cudaErrorInvalidValue;
  dot_partial_kernel<<<n_partial, kObjThreads, 0, s>>>(W, P, (long long)V * Kp, partial);
  return cudaGetLastError();
}

cudaError_t objective_finish(int Kp, const float* S, const float* Q, double normA2, double* partial,
                             int n_partial, double* out, unsigned* d_counter, int hist_cap, cudaStream_t s,
                             double* last) {
  if (Kp & 3) return cudaErrorInvalidValue;
  dot_partial_kernel<<<kSqBlocks, kObjThreads, 0, s>>>(S, Q, (long long)Kp * Kp, partial + n_partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  objective_final_kernel<<<1, kObjThreads, 0, s>>>(partial, n_partial, kSqBlocks, normA2, out, d_counter, hist_cap,
                                                    last);
  return cudaGetLastError();
}

cudaError_t objective_run(const float* W, const float* P, int V, int Kp, const float* S, const float* Q,
                          double normA2, double* partial, int n_partial, double* out, unsigned* d_counter,
                          int hist_cap, cudaStream_t s) {
  cudaError_t e = objective_wp(W, P, V, Kp, partial, n_partial, s);
  if (e != cudaSuccess) return e;
  return objective_finish(Kp, S, Q, normA2, partial, n_partial, out, d_counter, hist_cap, s);
}

// d_out must hold kSumsqBlocks doubles; the host adds them in order.
cudaError_t sumsq_dense_f64(const float* A, int64_t rows, int64_t cols, int64_t ld, double* d_out, int* d_bad,
                            cudaStream_t s) {
  sumsq_dense_kernel<<<kSumsqBlocks, 256, 0, s>>>(A, rows, cols, ld, d_out, d_bad);
  return cudaGetLastError();
}

}  // namespace plnmf
