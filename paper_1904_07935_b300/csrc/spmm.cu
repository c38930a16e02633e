// CSR SpMM for the products P = A H^T and R = A^T W (the products of Alg. 1)
// when A is a sparse term-document matrix (the paper calls a library CSR
// routine there, Sec. 4.1 / 4.2).
//
// Work plan (built once on the host): every CSR row becomes one work item,
// except rows longer than `seg` non-zeros (the Zipf head words, which can hold
// nearly every document), which are cut into items of at most `seg`
// non-zeros.  A warp owns an item (see spmm_items_kernel for the lane
// layout); the gathered rows of X are read as 16-byte loads.  The items of a
// split row write partial rows to a scratch buffer; the one that finishes
// last (a per-row counter) adds them in slot order, so results are
// bit-reproducible (no floating-point atomics) and no second launch is
// needed.  Items are ordered longest first to balance the tail.
#include <algorithm>
#include <numeric>

#include "devutil.cuh"
#include "internal.cuh"

namespace plnmf {
namespace {

// acc += a x, two lanes per packed FP32 multiply-add (each half rounded as
// a scalar fmaf).
__device__ __forceinline__ void fma4(float4& acc, float a, const float4& x) {
  const float2 aa = make_float2(a, a);
  fma_pair(acc.x, acc.y, aa, make_float2(x.x, x.y));
  fma_pair(acc.z, acc.w, aa, make_float2(x.z, x.w));
}

// Minimum resident CTAs per SM the compiler plans registers for.  It bounds
// the registers, and with them how many gathers a thread keeps in flight,
// while the occupancy stays what the 256-thread CTAs get anyway.  Measured on
// the text-like matrix against the compiler's default (52-60 registers):
// three CTAs from 5 to 6 chunks, two at 8 (K = 160: R 82 -> 54 us,
// P 79 -> 53 us; K = 400: R 300 -> 103 us, P 270 -> 109 us).  The 4-chunk
// layouts (K <= 64 and 97 <= K <= 128, the sizes of the batched workload's
// members) keep the compiler's own choice (44 registers): there many
// members' kernels share the SMs, and three planned CTAs (66 registers) cost
// the batch of 64 3% (20.8k against 21.5k instance-iterations per second).
constexpr int spmm_min_blocks(int C) { return C >= 8 ? 2 : 3; }

// One warp per work item.  The warp is split into G = 32 / L groups of L
// lanes; group g takes non-zeros beg + g, beg + g + G, ... and each of its
// lanes owns C float4 chunks of the output row (L * C * 4 >= Kp), so one step
// gathers G rows of X at once with 16-byte loads (two steps in flight).  At
// the end the G group sums are added with shuffles in a fixed tree order.
template <int L, int C>
__device__ __forceinline__ void spmm_items(const int4* __restrict__ items, int n_items,
                                           const int* __restrict__ col_idx, const float* __restrict__ val,
                                           const float4* __restrict__ X, int Kp4, float4* __restrict__ Y,
                                           float4* __restrict__ partial, const int4* __restrict__ comb,
                                           const int* __restrict__ slot_long, int* __restrict__ counter) {
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31;
  const int g = lane / L, sub = lane % L;
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (item >= n_items) return;                     // whole warp leaves together
  const int4 it = items[item];

  float4 acc[C];
#pragma unroll
  for (int q = 0; q < C; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);

  int e = it.y + g;
  for (; e + G < it.z; e += 2 * G) {               // two non-zeros per group in flight
    const int c0 = __ldg(col_idx + e), c1 = __ldg(col_idx + e + G);
    const float a0 = __ldg(val + e), a1 = __ldg(val + e + G);
    const float4* x0 = X + (size_t)c0 * Kp4;
    const float4* x1 = X + (size_t)c1 * Kp4;
    float4 v0[C], v1[C];
#pragma unroll
    for (int q = 0; q < C; ++q) {
      const int k = sub + L * q;
      v0[q] = k < Kp4 ? __ldg(x0 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      v1[q] = k < Kp4 ? __ldg(x1 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < C; ++q) {
      fma4(acc[q], a0, v0[q]);
      fma4(acc[q], a1, v1[q]);
    }
  }
  if (e < it.z) {
    const int c0 = __ldg(col_idx + e);
    const float a0 = __ldg(val + e);
    const float4* x0 = X + (size_t)c0 * Kp4;
#pragma unroll
    for (int q = 0; q < C; ++q) {
      const int k = sub + L * q;
      if (k < Kp4) fma4(acc[q], a0, __ldg(x0 + k));
    }
  }
  // Add the group sums: xor-shuffles over the group index bits.
#pragma unroll
  for (int off = L; off < 32; off <<= 1) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
      acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, off);
      acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, off);
      acc[q].z += __shfl_xor_sync(0xffffffffu, acc[q].z, off);
      acc[q].w += __shfl_xor_sync(0xffffffffu, acc[q].w, off);
    }
  }
  float4* dst = (it.w < 0) ? (Y + (size_t)it.x * Kp4) : (partial + (size_t)it.w * Kp4);
  if (g == 0) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
      const int k = sub + L * q;
      if (k < Kp4) dst[k] = acc[q];
    }
  }
  if (it.w < 0) return;                            // whole warp: a row of its own
  // Split row: the item that finishes last adds the row's partials in slot
  // order (each partial written and fenced before its item is counted).
  __threadfence();
  __syncwarp();
  const int lr = slot_long[it.w];
  const int4 c = comb[lr];
  int last = 0;
  if (lane == 0) last = atomicAdd(counter + lr, 1) == c.z - 1;
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
  for (int k = lane; k < Kp4; k += 32) {
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < c.z; ++j) {
      const float4 v = __ldcg(partial + (size_t)(c.y + j) * Kp4 + k);
      sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
    }
    Y[(size_t)c.x * Kp4 + k] = sum;
  }
  if (lane == 0) counter[lr] = 0;                  // ready for the next launch
}

template <int L, int C>
__global__ void __launch_bounds__(256, spmm_min_blocks(C))
    spmm_items_kernel(const int4* __restrict__ items, int n_items, const int* __restrict__ col_idx,
                      const float* __restrict__ val, const float4* __restrict__ X, int Kp4, float4* __restrict__ Y,
                      float4* __restrict__ partial, const int4* __restrict__ comb,
                      const int* __restrict__ slot_long, int* __restrict__ counter) {
  spmm_items<L, C>(items, n_items, col_idx, val, X, Kp4, Y, partial, comb, slot_long, counter);
}
template <int L, int C>
__global__ void __launch_bounds__(256)
    spmm_items_lean_kernel(const int4* __restrict__ items, int n_items, const int* __restrict__ col_idx,
                           const float* __restrict__ val, const float4* __restrict__ X, int Kp4,
                           float4* __restrict__ Y, float4* __restrict__ partial, const int4* __restrict__ comb,
                           const int* __restrict__ slot_long, int* __restrict__ counter) {
  spmm_items<L, C>(items, n_items, col_idx, val, X, Kp4, Y, partial, comb, slot_long, counter);
}

template <int L, int C>
cudaError_t launch_items(const SpmmPlan& p, const int* ci, const float* va, const float* X, float* Y,
                         int Kp, cudaStream_t s) {
  const int Kp4 = Kp / 4;
  const int warps_per_block = 8;
  const int blocks = (p.n_items + warps_per_block - 1) / warps_per_block;
  if (blocks > 0) {
    const float4* x4 = reinterpret_cast<const float4*>(X);
    float4* y4 = reinterpret_cast<float4*>(Y);
    float4* p4 = reinterpret_cast<float4*>(p.d_partial);
    if constexpr (C == 4) {
      spmm_items_lean_kernel<L, C><<<blocks, 32 * warps_per_block, 0, s>>>(
          p.d_items, p.n_items, ci, va, x4, Kp4, y4, p4, p.d_combine, p.d_slot_long, p.d_counter);
    } else {
      spmm_items_kernel<L, C><<<blocks, 32 * warps_per_block, 0, s>>>(
          p.d_items, p.n_items, ci, va, x4, Kp4, y4, p4, p.d_combine, p.d_slot_long, p.d_counter);
    }
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
  std::vector<int> slot_long((size_t)std::max(1, slot), 0);
  for (size_t i = 0; i < comb.size(); ++i)
    for (int j = 0; j < comb[i].z; ++j) slot_long[(size_t)comb[i].y + j] = (int)i;
  if ((err = cudaMalloc(&plan.d_slot_long, sizeof(int) * slot_long.size())) != cudaSuccess) return err;
  if ((err = cudaMemcpy(plan.d_slot_long, slot_long.data(), sizeof(int) * slot_long.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess) return err;
  if ((err = cudaMalloc(&plan.d_counter, sizeof(int) * std::max<size_t>(1, comb.size()))) != cudaSuccess) return err;
  if ((err = cudaMemset(plan.d_counter, 0, sizeof(int) * std::max<size_t>(1, comb.size()))) != cudaSuccess) return err;
  return cudaDeviceSynchronize();
}

void spmm_plan_free(SpmmPlan& plan) {
  cudaFree(plan.d_items);
  cudaFree(plan.d_combine);
  cudaFree(plan.d_partial);
  cudaFree(plan.d_slot_long);
  cudaFree(plan.d_counter);
  plan.d_items = nullptr;
  plan.d_combine = nullptr;
  plan.d_partial = nullptr;
  plan.d_slot_long = nullptr;
  plan.d_counter = nullptr;
}

cudaError_t spmm_run(const SpmmPlan& p, const int* ci, const float* va, const float* X, float* Y,
                     int Kp, cudaStream_t s) {
  const int Kp4 = Kp / 4;
  cudaError_t err;
  // Lanes per non-zero L and float4 chunks per lane C with L * C >= Kp / 4,
  // chosen to keep C <= 8 and few idle chunks.
  if (Kp4 <= 4) err = launch_items<1, 4>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 8) err = launch_items<2, 4>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 16) err = launch_items<4, 4>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 20) err = launch_items<4, 5>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 24) err = launch_items<4, 6>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 32) err = launch_items<8, 4>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 40) err = launch_items<8, 5>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 48) err = launch_items<8, 6>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 64) err = launch_items<8, 8>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 80) err = launch_items<16, 5>(p, ci, va, X, Y, Kp, s);
  else if (Kp4 <= 96) err = launch_items<16, 6>(p, ci, va, X, Y, Kp, s);
  else err = launch_items<16, 8>(p, ci, va, X, Y, Kp, s);   // Kp <= 512
  return err;
}

}  // namespace plnmf
