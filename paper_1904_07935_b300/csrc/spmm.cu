// CSR SpMM for the products P = A H^T and R = A^T W (Alg. 1, lines 4 and 10)
// when A is a sparse term-document matrix (the paper calls a library CSR
// routine there, Sec. 4.1 / 4.2).
//
// Work plan (built once on the host): every CSR row becomes one work item,
// except rows longer than `seg` non-zeros (the Zipf head words, which can hold
// nearly every document), which are cut into items of at most `seg`
// non-zeros.  A group of lanes owns an item: the lanes cover the Kp/4 float4
// chunks of one output row, the non-zeros are streamed 32 at a time and
// broadcast with shuffles, and the gathered rows of X are read as float4
// (coalesced 16-byte loads).  Split rows write partial rows to a scratch
// buffer and a second kernel adds them in a fixed order, so results are
// bit-reproducible (no floating-point atomics).  Items are ordered longest
// first to balance the tail.
#include <algorithm>
#include <numeric>

#include "internal.cuh"

namespace plnmf {
namespace {

__device__ __forceinline__ void fma4(float4& acc, float a, const float4& x) {
  acc.x = fmaf(a, x.x, acc.x);
  acc.y = fmaf(a, x.y, acc.y);
  acc.z = fmaf(a, x.z, acc.z);
  acc.w = fmaf(a, x.w, acc.w);
}

// LPR lanes per item (power of two <= 32), VPL float4 chunks per lane.
template <int LPR, int VPL>
__global__ void __launch_bounds__(256) spmm_items_kernel(const int4* __restrict__ items, int n_items,
                                                         const int* __restrict__ col_idx,
                                                         const float* __restrict__ val,
                                                         const float4* __restrict__ X, int Kp4,
                                                         float4* __restrict__ Y,
                                                         float4* __restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LPR - 1);                 // lane inside the item group
  const int group = (blockIdx.x * blockDim.x + threadIdx.x) / LPR;
  const bool active = group < n_items;
  int4 it = active ? items[group] : make_int4(0, 0, 0, -1);
  const unsigned full = 0xffffffffu;

  float4 acc[VPL];
#pragma unroll
  for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);

  // Every lane of the warp must take part in the shuffles, so the loop runs
  // to the longest item in the warp; shorter groups see n = 0.
  int beg = it.y, end = active ? it.z : it.y;
  for (int e0 = beg;; e0 += LPR) {
    const int remaining = end - e0;
    const int any = __any_sync(full, remaining > 0);
    if (!any) break;
    int c = 0;
    float a = 0.f;
    if (sub < remaining) {
      c = __ldg(col_idx + e0 + sub);
      a = __ldg(val + e0 + sub);
    }
    const int n = max(0, min(LPR, remaining));
#pragma unroll 4
    for (int j = 0; j < LPR; ++j) {
      const int cj = __shfl_sync(full, c, j, LPR);
      const float aj = __shfl_sync(full, a, j, LPR);
      if (j < n) {
        const float4* xr = X + (size_t)cj * Kp4;
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
          const int idx = sub + LPR * q;
          if (idx < Kp4) fma4(acc[q], aj, __ldg(xr + idx));
        }
      }
    }
  }
  if (!active) return;
  float4* dst = (it.w < 0) ? (Y + (size_t)it.x * Kp4) : (partial + (size_t)it.w * Kp4);
#pragma unroll
  for (int q = 0; q < VPL; ++q) {
    const int idx = sub + LPR * q;
    if (idx < Kp4) dst[idx] = acc[q];
  }
}

// Y[row] = sum of its partial rows in slot order.
__global__ void spmm_combine_kernel(const int4* __restrict__ comb, int n_long,
                                    const float4* __restrict__ partial, float4* __restrict__ Y,
                                    int Kp4) {
  const int i = blockIdx.x;
  if (i >= n_long) return;
  const int4 c = comb[i];
  for (int k = threadIdx.x; k < Kp4; k += blockDim.x) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < c.z; ++j) {
      const float4 p = partial[(size_t)(c.y + j) * Kp4 + k];
      s.x += p.x; s.y += p.y; s.z += p.z; s.w += p.w;
    }
    Y[(size_t)c.x * Kp4 + k] = s;
  }
}

template <int LPR, int VPL>
cudaError_t launch_items(const SpmmPlan& p, const int* ci, const float* va, const float* X, float* Y,
                         int Kp, cudaStream_t s) {
  const int Kp4 = Kp / 4;
  const int per_block = 256 / LPR;
  const int blocks = (p.n_items + per_block - 1) / per_block;
  if (blocks > 0) {
    spmm_items_kernel<LPR, VPL><<<blocks, 256, 0, s>>>(
        p.d_items, p.n_items, ci, va, reinterpret_cast<const float4*>(X), Kp4,
        reinterpret_cast<float4*>(Y), reinterpret_cast<float4*>(p.d_partial));
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t spmm_plan_build(SpmmPlan& plan, const std::vector<int>& row_ptr, int rows, int cols,
                            int Kp, int seg) {
  plan.rows = rows;
  plan.cols = cols;
  std::vector<int4> items;
  std::vector<int4> comb;
  std::vector<int4> long_items;
  int slot = 0;
  items.reserve(rows);
  for (int r = 0; r < rows; ++r) {
    const int b = row_ptr[r], e = row_ptr[r + 1];
    const int len = e - b;
    if (len <= seg) {
      items.push_back(make_int4(r, b, e, -1));
    } else {
      const int nseg = (len + seg - 1) / seg;
      comb.push_back(make_int4(r, slot, nseg, 0));
      for (int j = 0; j < nseg; ++j) {
        const int sb = b + j * seg;
        long_items.push_back(make_int4(r, sb, std::min(e, sb + seg), slot + j));
      }
      slot += nseg;
    }
  }
  // Longest items first (split segments are all `seg` long or a tail).
  std::stable_sort(items.begin(), items.end(),
                   [](const int4& a, const int4& b) { return (a.z - a.y) > (b.z - b.y); });
  long_items.insert(long_items.end(), items.begin(), items.end());
  plan.n_items = (int)long_items.size();
  plan.n_long = (int)comb.size();
  plan.n_slots = slot;
  cudaError_t err;
  if ((err = cudaMalloc(&plan.d_items, sizeof(int4) * std::max<size_t>(1, long_items.size()))) != cudaSuccess) return err;
  if ((err = cudaMemcpy(plan.d_items, long_items.data(), sizeof(int4) * long_items.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess) return err;
  if ((err = cudaMalloc(&plan.d_combine, sizeof(int4) * std::max<size_t>(1, comb.size()))) != cudaSuccess) return err;
  if (!comb.empty() &&
      (err = cudaMemcpy(plan.d_combine, comb.data(), sizeof(int4) * comb.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  if ((err = cudaMalloc(&plan.d_partial, sizeof(float) * (size_t)std::max(1, slot) * Kp)) != cudaSuccess) return err;
  return cudaSuccess;
}

void spmm_plan_free(SpmmPlan& plan) {
  cudaFree(plan.d_items);
  cudaFree(plan.d_combine);
  cudaFree(plan.d_partial);
  plan.d_items = nullptr;
  plan.d_combine = nullptr;
  plan.d_partial = nullptr;
}

cudaError_t spmm_run(const SpmmPlan& p, const int* ci, const float* va, const float* X, float* Y,
                     int Kp, cudaStream_t s) {
  const int Kp4 = Kp / 4;
  cudaError_t err;
  if (Kp4 <= 1) err = launch_items<1, 1>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 2) err = launch_items<2, 1>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 4) err = launch_items<4, 1>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 8) err = launch_items<8, 1>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 16) err = launch_items<16, 1>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 32) err = launch_items<32, 1>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 64) err = launch_items<32, 2>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 96) err = launch_items<32, 3>(p, ci, va, X, Y, Kp, s);
  else err = launch_items<32, 4>(p, ci, va, X, Y, Kp, s);   // Kp <= 512
  if (err != cudaSuccess) return err;
  if (p.n_long > 0) {
    spmm_combine_kernel<<<p.n_long, 128, 0, s>>>(p.d_combine, p.n_long,
                                                 reinterpret_cast<const float4*>(p.d_partial),
                                                 reinterpret_cast<float4*>(Y), Kp4);
    err = cudaGetLastError();
  }
  return err;
}

}  // namespace plnmf
