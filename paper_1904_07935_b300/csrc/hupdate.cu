// Fused H update (Alg. 1 lines 6-8 in the tiled order of Alg. 2).
//
// H carries no normalisation, so every document (row of H^T) is updated
// independently of the others (Sec. 4.1, last sentence) and the whole update
// is one launch: each row is owned by a group of 4 lanes, each lane owning 4
// of the 16 columns of the current tile.  For tile [lo, hi) and column c:
//   y_c = R[c] + (1 - S_cc) h_c - sum_{j < lo} S[j][c] h_j(new)
//                               - sum_{j >= hi} S[j][c] h_j(old)
//                               - sum_{c < j < hi} S[j][c] h_j(old)
// and then, inside the tile, column t is finished (clamped at eps) and
// broadcast to the lanes of its row, which subtract S[t][c] h_t(new) from
// their later columns (Eq. 5).  Earlier tiles are already written back, so
// row j < lo of the factor holds new values and j >= lo old ones: the
// contributions of Eqs. 4 and 6 are one pass over the row.
#include "internal.cuh"

namespace plnmf {
namespace {

constexpr int HT = 16;            // tile width
constexpr int HL = 4;             // lanes per row
constexpr int HROWS = 64;         // rows per CTA
constexpr int HTHREADS = HROWS * HL;

__global__ void __launch_bounds__(HTHREADS) h_update_kernel(float* __restrict__ X, const float* __restrict__ B,
                                                            const float* __restrict__ G, int N, int K, int Kp,
                                                            float eps) {
  extern __shared__ __align__(16) float Gc[];     // Kr x HT: G[j][lo + c], zero beyond K
  const int Kr = (Kp + HT - 1) / HT * HT;         // rows reachable as lo + t
  const int tid = threadIdx.x;
  const int sub = tid & (HL - 1);
  const int row = blockIdx.x * HROWS + (tid >> 2);
  const bool valid = row < N;
  const unsigned full = 0xffffffffu;
  float* xr = X + (int64_t)(valid ? row : 0) * Kp;
  const float* br = B + (int64_t)(valid ? row : 0) * Kp;

  for (int lo = 0; lo < K; lo += HT) {
    const int hi = min(K, lo + HT);
    __syncthreads();
    for (int e = tid; e < Kr * HT; e += HTHREADS) {
      const int j = e / HT, c = e % HT;
      Gc[e] = (j < K && lo + c < K) ? __ldg(G + (int64_t)j * Kp + lo + c) : 0.f;
    }
    __syncthreads();

    // Old values of this row's tile (all 16, shared by the 4 lanes).
    float xo[HT];
#pragma unroll
    for (int q = 0; q < HT / 4; ++q) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid && lo + 4 * q < Kp) v = *reinterpret_cast<const float4*>(xr + lo + 4 * q);
      xo[4 * q] = v.x; xo[4 * q + 1] = v.y; xo[4 * q + 2] = v.z; xo[4 * q + 3] = v.w;
    }
    // Columns of this lane: lo + 4 * sub + q (its own old values read again
    // so that no register array is indexed by the lane number).
    float acc[4];
    float4 own = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid && lo + 4 * sub < Kp) own = *reinterpret_cast<const float4*>(xr + lo + 4 * sub);
    const float xown[4] = {own.x, own.y, own.z, own.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cl = 4 * sub + q, c = lo + cl;
      acc[q] = 0.f;
      if (valid && c < hi) {
        const float gcc = Gc[c * HT + cl];
        acc[q] = fmaf(1.f - gcc, xown[q], br[c]);
      }
    }
    // Columns outside the tile: j < lo (new) and j >= hi (old); padding
    // columns of X and rows of G are zero, so the loop runs to Kp.
    auto outside = [&](int j0, int j1) {
      for (int j = j0; j < j1; j += 4) {
        const float4 x4 = valid ? *reinterpret_cast<const float4*>(xr + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 g = *reinterpret_cast<const float4*>(Gc + (j + u) * HT + 4 * sub);
          acc[0] = fmaf(-g.x, xs[u], acc[0]);
          acc[1] = fmaf(-g.y, xs[u], acc[1]);
          acc[2] = fmaf(-g.z, xs[u], acc[2]);
          acc[3] = fmaf(-g.w, xs[u], acc[3]);
        }
      }
    };
    outside(0, lo);
    outside(lo + HT < Kp ? lo + HT : Kp, Kp);
    // Old in-tile columns j > c.
#pragma unroll
    for (int j = 1; j < HT; ++j) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cl = 4 * sub + q;
        if (j > cl) acc[q] = fmaf(-Gc[(lo + j) * HT + cl], xo[j], acc[q]);
      }
    }
    // Finish the tile's columns in order; each new value is broadcast to the
    // row's lanes and pushed into the later columns.
    float xn[4];
#pragma unroll
    for (int t = 0; t < HT; ++t) {
      const int owner = t >> 2, q = t & 3;
      float v = 0.f;
      if (sub == owner) {
        v = fmaxf(eps, acc[q]);
        xn[q] = v;
      }
      v = __shfl_sync(full, v, (threadIdx.x & 31 & ~(HL - 1)) + owner);
#pragma unroll
      for (int q2 = 0; q2 < 4; ++q2) {
        const int c2 = 4 * sub + q2;
        if (c2 > t) acc[q2] = fmaf(-Gc[(lo + t) * HT + c2], v, acc[q2]);
      }
    }
    if (valid) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lo + 4 * sub + q;
        if (c < hi) xr[c] = xn[q];
      }
    }
  }
}

}  // namespace

cudaError_t h_update_run(float* X, const float* B, const float* G, int N, int K, int Kp, float eps,
                         cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)((Kp + HT - 1) / HT * HT) * HT;
  cudaError_t e = cudaFuncSetAttribute(h_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (N + HROWS - 1) / HROWS;
  h_update_kernel<<<blocks, HTHREADS, smem, s>>>(X, B, G, N, K, Kp, eps);
  return cudaGetLastError();
}

}  // namespace plnmf
