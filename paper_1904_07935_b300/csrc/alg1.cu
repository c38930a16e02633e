// Comparator: HALS without column tiling (Sec. 3).  Each factor is updated
// one column at a time, every column being the exact non-negative minimiser
// of the objective in that column with all others fixed, and columns taken in
// ascending order so that column k sees the new values of columns < k.  For
// the tall factor X with data term B and Gram G (H: X = H^T, B = R, G = S;
// W: X = W, B = P, G = Q):
//   x_k <- max(eps, x_k G_kk + B_k - X G_k)     (W; then x_k <- x_k / ||x_k||)
//   x_k <- max(eps, x_k + B_k - X G_k)          (H, where G_kk = 1 by the unit
//                                                 columns of W)
// X G_k is the product with the current X (columns < k already new,
// including the k-th term).  Without tiling there is no cheaper way to form
// it than a pass over the whole factor per column: one warp per row, column
// k one grid-wide launch (W: a second launch normalises the column before
// the next one reads it), K (H) or 2K (W) dependent launches per update.
// This is what the tiled order of Sec. 4 (Eqs. 4-6) is measured against.
// G is symmetric, so column k is read as row k (contiguous).
#include "devutil.cuh"
#include "internal.cuh"

namespace plnmf {
namespace {

constexpr int kWarps = 8;                // warps (rows) per CTA

// Row d of X (N x Kp) dotted with row k of G (the Gram, K x Kp), lanes
// striding the K terms, summed by a fixed xor tree (every lane gets it).
__device__ __forceinline__ float row_dot(const float* __restrict__ x, const float* __restrict__ g, int K) {
  const int lane = threadIdx.x & 31;
  float s = 0.f;
  for (int j = lane; j < K; j += 32) s = fmaf(x[j], g[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__global__ void __launch_bounds__(32 * kWarps) alg1_h_column_kernel(float* __restrict__ Ht, const float* __restrict__ R,
                                                                   const float* __restrict__ S, int D, int K, int Kp,
                                                                   int k, float eps) {
  const int d = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (d >= D) return;                                      // whole warp
  float* h = Ht + (int64_t)d * Kp;
  const float dot = row_dot(h, S + (int64_t)k * Kp, K);
  if ((threadIdx.x & 31) == 0) h[k] = fmaxf(eps, h[k] + R[(int64_t)d * Kp + k] - dot);
}

// New (unnormalised) w_k for this CTA's rows, and the CTA's sum of squares
// (fixed order) in part[blockIdx.x].
__global__ void __launch_bounds__(32 * kWarps) alg1_w_column_kernel(float* __restrict__ W, const float* __restrict__ P,
                                                                   const float* __restrict__ Q, int V, int K, int Kp,
                                                                   int k, float eps, float* __restrict__ part) {
  __shared__ float sq[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * kWarps + warp;
  float w = 0.f;
  if (v < V) {
    float* x = W + (int64_t)v * Kp;
    const float dot = row_dot(x, Q + (int64_t)k * Kp, K);
    w = fmaxf(eps, fmaf(x[k], Q[(int64_t)k * Kp + k], P[(int64_t)v * Kp + k]) - dot);
    if (lane == 0) x[k] = w;
  }
  if (lane == 0) sq[warp] = v < V ? w * w : 0.f;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) s += sq[i];
    part[blockIdx.x] = s;
  }
}

// Every CTA adds all n_part partial sums in the same fixed order (so every
// CTA gets the same norm; compensated) and scales its rows of column k.
__global__ void __launch_bounds__(256) alg1_w_scale_kernel(float* __restrict__ W, int V, int Kp, int k,
                                                          const float* __restrict__ part, int n_part,
                                                          int* __restrict__ status) {
  __shared__ float ss[256], sc[256];
  float s = 0.f, c = 0.f;
  for (int i = threadIdx.x; i < n_part; i += 256) {
    float e;
    two_sum(s, part[i], s, e);
    c += e;
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      float e;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + off], ss[threadIdx.x], e);
      sc[threadIdx.x] += sc[threadIdx.x + off] + e;
    }
    __syncthreads();
  }
  const float tot = ss[0] + sc[0];
  const float nrm = sqrtf(tot);
  if (blockIdx.x == 0 && threadIdx.x == 0 && (!(nrm > 0.f) || !(nrm < INFINITY))) atomicOr(status, ST_NUMERIC);
  const float inv = 1.0f / nrm;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
    W[(int64_t)v * Kp + k] *= inv;
}

}  // namespace

int alg1_parts(int V) { return (V + kWarps - 1) / kWarps; }

cudaError_t alg1_update_h(float* Ht, const float* R, const float* S, int D, int K, int Kp, float eps,
                          cudaStream_t s, int* launches) {
  const int blocks = (D + kWarps - 1) / kWarps;
  for (int k = 0; k < K; ++k) {
    alg1_h_column_kernel<<<blocks, 32 * kWarps, 0, s>>>(Ht, R, S, D, K, Kp, k, eps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches += K;
  return cudaSuccess;
}

cudaError_t alg1_update_w(float* W, const float* P, const float* Q, int V, int K, int Kp, float eps, float* part,
                          int* status, cudaStream_t s, int* launches) {
  const int blocks = alg1_parts(V);
  const int sblocks = std::min(148, (V + 255) / 256);
  for (int k = 0; k < K; ++k) {
    alg1_w_column_kernel<<<blocks, 32 * kWarps, 0, s>>>(W, P, Q, V, K, Kp, k, eps, part);
    alg1_w_scale_kernel<<<sblocks, 256, 0, s>>>(W, V, Kp, k, part, blocks, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches += 2 * K;
  return cudaSuccess;
}

}  // namespace plnmf
