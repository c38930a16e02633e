// Multiplicative updates (Lee & Seung 2001), the comparator the paper sets
// PL-NMF against (Sec. 2, Sec. 6):
//   H <- H * (W^T A) / (W^T W H + delta),  W <- W * (A H^T) / (W H H^T + delta)
// in the tall layout: Ht <- Ht * R / (Ht S + delta), W <- W * P / (W Q + delta)
// (S and Q symmetric).  The products are the library's; this file holds the
// elementwise step.
#include "internal.cuh"

namespace plnmf {
namespace {

// X[r][c] *= B[r][c] / (C[r][c] + delta) for c < K (row stride Kp; the
// padding columns stay zero).  16-byte accesses, grid-stride.
__global__ void mu_scale_kernel(float* __restrict__ X, const float* __restrict__ B, const float* __restrict__ C,
                                int64_t n4, int Kp4, int K, float delta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const int c0 = (int)(i % Kp4) * 4;
    float4 x = reinterpret_cast<float4*>(X)[i];
    const float4 b = reinterpret_cast<const float4*>(B)[i];
    const float4 d = reinterpret_cast<const float4*>(C)[i];
    if (c0 < K) x.x *= b.x / (d.x + delta);
    if (c0 + 1 < K) x.y *= b.y / (d.y + delta);
    if (c0 + 2 < K) x.z *= b.z / (d.z + delta);
    if (c0 + 3 < K) x.w *= b.w / (d.w + delta);
    reinterpret_cast<float4*>(X)[i] = x;
  }
}

}  // namespace

cudaError_t mu_update(float* X, const float* B, const float* G, float* scratch, int N, int K, int Kp, float delta,
                      cudaStream_t s, int* launches) {
  GemmArgs a;
  a.M = N;
  a.N = Kp;
  a.Kin = Kp;
  a.A = X;
  a.lda = Kp;
  a.transA = 0;
  a.B = G;
  a.ldb = Kp;
  a.transB = 0;
  a.C = scratch;
  a.ldc = Kp;
  a.mode = GM_STORE;
  cudaError_t e = gemm_run(a, s);                            // scratch = X G
  if (e != cudaSuccess) return e;
  const int64_t n4 = (int64_t)N * (Kp / 4);
  const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 148 * 8);
  mu_scale_kernel<<<blocks, 256, 0, s>>>(X, B, scratch, n4, Kp / 4, K, delta);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

}  // namespace plnmf
