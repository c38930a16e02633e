// Phase 2 of the regrouped factor update (Alg. 2 inner loop, Eq. 5): the
// columns of one tile are finished one after another.
//
// On entry Y[:, lo:hi] holds, for every row v and column t of the tile,
//   B[v,t] + c'_t X_old[v,t] - sum_{j > t} G[j,t] X_old[v,j]
//                            - sum_{j < lo} G[j,t] X_new[v,j]
// (phase 1 and the phase-3 updates of earlier tiles).  The kernel adds the
// remaining contributions of new columns inside the tile, clamps at eps and,
// for W, divides every finished column by its L2 norm before the next column
// uses it (Alg. 1 lines 13-15).  Each thread keeps its rows' tile of Y in
// registers; when column t is final its value is pushed into the later
// columns of the tile ("right-looking"), so a column costs one clamp, one
// square and the norm reduction on the critical path.
//
// The norm needs every row, so the W chain runs on one thread-block cluster
// (16 CTAs where the GPU allows, else 8): each CTA reduces its rows (warp
// shuffles, then one warp over the per-warp sums) and sends its partial to
// every CTA of the cluster with st.async into distributed shared memory,
// completing a transaction count on the receiver's mbarrier.  Every CTA then
// adds the CL partials in rank order, so all CTAs (and all runs) see the same
// norm.  Two slots alternate between consecutive columns.  Every wait is
// bounded; on expiry the kernel sets ST_TIMEOUT and stops waiting.
//
// The H update (no normalisation, rows independent) uses the same kernel
// without the cluster reduction on a grid covering all rows.
#include <algorithm>

#include "internal.cuh"

namespace plnmf {
namespace {

struct ChainParams {
  float* Y;
  float* X;
  const float* G;
  int N, Kp, lo, hi;
  float eps;
  int* status;
  int cl;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned mapa_u32(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void st_async_f32(unsigned raddr, float v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(raddr),
               "r"(__float_as_uint(v)), "r"(rbar)
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kMaxCluster = 16;
constexpr int kNormThreads = 256;
constexpr int kPlainThreads = 256;
constexpr int TT = kMaxChainTile;        // register tile width (columns)

// Output buffer of the finished columns: st[(i * TT + t) * (NT + 1) + r]
// holds column t of thread-row r in row group i.
template <int NT>
__device__ __forceinline__ int st_idx(int i, int t, int r) {
  return (i * TT + t) * (NT + 1) + r;
}

// Each thread keeps RPT rows of the tile in registers, y[i][0..TT).  Column t
// of the tile is always in slot 0: when it is final, its value x is pushed into
// the later columns and the row shifts left in the same fused multiply-add,
//   y[i][c - 1] = y[i][c] - x * G[lo + t][lo + t + c],
// so every register index is static and the column loop stays a loop.
template <int NT, int RPT, bool NORM>
__global__ void __launch_bounds__(NT) chain_kernel(ChainParams p) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) float st[];    // RPT x TT x (NT + 1)
  __shared__ float Gs[TT][2 * TT];               // G block, zero beyond the tile
  __shared__ float wpart[NW];
  __shared__ float cpart[2][kMaxCluster];
  __shared__ float col_inv;
  __shared__ __align__(8) unsigned long long mbar[2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Tw = p.hi - p.lo;
  const unsigned rank = NORM ? cluster_ctarank() : blockIdx.x;
  const int CL = NORM ? p.cl : (int)gridDim.x;

  for (int e = tid; e < TT * 2 * TT; e += NT) {
    const int i = e / (2 * TT), j = e % (2 * TT);
    Gs[i][j] = (i < Tw && j < Tw) ? p.G[(int64_t)(p.lo + i) * p.Kp + p.lo + j] : 0.f;
  }
  if (NORM && tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    // Expect the first two columns' partials before anyone can send them.
    mbar_arrive_expect_tx(smem_u32(&mbar[0]), CL * 4);
    if (Tw > 1) mbar_arrive_expect_tx(smem_u32(&mbar[1]), CL * 4);
    fence_mbar_init();
  }

  // Rows: thread-row r of row group i is row (rank * NT + r) + i * CL * NT.
  // Each thread reads its own rows' tile: 16-byte loads when the tile starts
  // on a 16-byte boundary, scalar loads otherwise; all loads of a thread are
  // independent, so they overlap.
  const int cta_base = (int)rank * NT;
  const int stride = CL * NT;
  const bool vec = (p.lo & 3) == 0;
  float y[RPT][TT];
  bool valid[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int row = cta_base + tid + i * stride;
    valid[i] = row < p.N;
    const float* src = p.Y + (int64_t)(valid[i] ? row : 0) * p.Kp + p.lo;
#pragma unroll
    for (int q = 0; q < TT / 4; ++q) {
      if (valid[i] && vec && 4 * q + 3 < Tw) {
        const float4 v = *reinterpret_cast<const float4*>(src + 4 * q);
        y[i][4 * q] = v.x; y[i][4 * q + 1] = v.y; y[i][4 * q + 2] = v.z; y[i][4 * q + 3] = v.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) y[i][4 * q + j] = (valid[i] && 4 * q + j < Tw) ? src[4 * q + j] : 0.f;
      }
    }
  }
  __syncthreads();
  if (NORM) cluster_sync_all();

  bool dead = false;
#pragma unroll 1
  for (int t = 0; t < Tw; ++t) {
    float x[RPT];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      x[i] = fmaxf(p.eps, y[i][0]);
      if (valid[i]) ss = fmaf(x[i], x[i], ss);
    }
    if (NORM) {
      const int b = t & 1;
      ss = warp_sum(ss);
      if (lane == 0) wpart[warp] = ss;
      __syncthreads();
      if (warp == 0) {
        float v = lane < NW ? wpart[lane] : 0.f;
        v = warp_sum(v);
        if (lane < CL) {
          const unsigned raddr = mapa_u32(smem_u32(&cpart[b][rank]), lane);
          const unsigned rbar = mapa_u32(smem_u32(&mbar[b]), lane);
          st_async_f32(raddr, v, rbar);
        }
        // Warp 0 waits for the CL partials; the barrier below releases the CTA.
        if (!dead) {
          const unsigned bar = smem_u32(&mbar[b]);
          const unsigned parity = (t >> 1) & 1;
          unsigned long long t0 = 0;
          unsigned polls = 0;
          while (!mbar_try_wait(bar, parity)) {
            if ((++polls & 31u) == 0) {
              const unsigned long long now = global_ns();
              if (t0 == 0) {
                t0 = now;
              } else if (now - t0 > kWaitLimitNs) {
                dead = true;
                if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
                break;
              }
            }
          }
        }
        dead = __any_sync(0xffffffffu, dead);
        // Sum of the CL partials as a fixed shuffle tree (the same order in
        // every CTA, so every CTA sees the same norm).
        float tot = lane < CL ? cpart[b][lane] : 0.f;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
        if (lane == 0) {
          const float nrm = sqrtf(tot);
          col_inv = 1.0f / nrm;
          if (t + 2 < Tw && !dead) mbar_arrive_expect_tx(smem_u32(&mbar[b]), CL * 4);
          if (!(nrm > 0.f) || !(nrm < INFINITY)) {
            if (rank == 0) atomicOr(p.status, ST_NUMERIC);
          }
        }
      }
      __syncthreads();
      const float inv = col_inv;
#pragma unroll
      for (int i = 0; i < RPT; ++i) x[i] *= inv;
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) st[st_idx<NT>(i, t, tid)] = x[i];
    // New column t contributes to the later columns of the tile; shift left.
#pragma unroll
    for (int c = 1; c < TT; ++c) {
      const float g = Gs[t][t + c];
#pragma unroll
      for (int i = 0; i < RPT; ++i) y[i][c - 1] = fmaf(-x[i], g, y[i][c]);
    }
  }
  // Each thread writes its own rows back (the staging buffer holds them in
  // column order for this thread, so the reads are conflict-free).
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    if (!valid[i]) continue;
    float* dst = p.X + (int64_t)(cta_base + tid + i * stride) * p.Kp + p.lo;
#pragma unroll
    for (int q = 0; q < TT / 4; ++q) {
      if (vec && 4 * q + 3 < Tw) {
        float4 v;
        v.x = st[st_idx<NT>(i, 4 * q, tid)];
        v.y = st[st_idx<NT>(i, 4 * q + 1, tid)];
        v.z = st[st_idx<NT>(i, 4 * q + 2, tid)];
        v.w = st[st_idx<NT>(i, 4 * q + 3, tid)];
        *reinterpret_cast<float4*>(dst + 4 * q) = v;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j < Tw) dst[4 * q + j] = st[st_idx<NT>(i, 4 * q + j, tid)];
      }
    }
  }
  // No CTA may leave while a peer can still write into its shared memory.
  if (NORM) cluster_sync_all();
}

size_t chain_smem_bytes(int rpt, int nt) { return sizeof(float) * (size_t)rpt * TT * (nt + 1); }

template <int RPT>
cudaError_t launch_norm_t(const ChainParams& p, cudaStream_t s) {
  auto kern = chain_kernel<kNormThreads, RPT, true>;
  const size_t smem = chain_smem_bytes(RPT, kNormThreads);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.cl > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.cl, 1, 1);
  cfg.blockDim = dim3(kNormThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = p.cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

cudaError_t launch_norm(const ChainParams& p, int rpt, cudaStream_t s) {
  switch (rpt) {
    case 1: return launch_norm_t<1>(p, s);
    case 2: return launch_norm_t<2>(p, s);
    case 3: return launch_norm_t<3>(p, s);
    case 4: return launch_norm_t<4>(p, s);
    case 5: return launch_norm_t<5>(p, s);
    case 6: return launch_norm_t<6>(p, s);
    case 7: return launch_norm_t<7>(p, s);
    case 8: return launch_norm_t<8>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_plain(const ChainParams& p, cudaStream_t s) {
  const int blocks = std::max(1, (p.N + kPlainThreads - 1) / kPlainThreads);
  const size_t smem = chain_smem_bytes(1, kPlainThreads);
  auto kern = chain_kernel<kPlainThreads, 1, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kPlainThreads, smem, s>>>(p);
  return cudaGetLastError();
}

int max_cluster_for(int rpt) {
  const size_t smem = chain_smem_bytes(rpt, kNormThreads);
  auto kern = chain_kernel<kNormThreads, 8, true>;   // largest variant bounds the others
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int cl : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl, 1, 1);
    cfg.blockDim = dim3(kNormThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0) return cl;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace

// Chooses the cluster size and rows per thread (at most 8 rows of 16 columns
// per thread, 256 threads per CTA).
bool chain_config_for(int N, bool normalize, int T, ChainConfig* cfg) {
  if (T < 1 || T > kMaxChainTile) return false;
  if (!normalize) {
    cfg->cluster = 1;
    cfg->threads = kPlainThreads;
    cfg->rpt = 1;
    cfg->tt = T;
    return true;
  }
  for (int cl : {16, 8}) {
    const int rpt = (N + cl * kNormThreads - 1) / (cl * kNormThreads);
    if (rpt > 8) continue;
    if (max_cluster_for(rpt) < cl) continue;
    cfg->cluster = cl;
    cfg->threads = kNormThreads;
    cfg->rpt = rpt;
    cfg->tt = T;
    return true;
  }
  return false;
}

cudaError_t chain_run(float* Y, float* X, const float* G, int N, int Kp, int lo, int hi, float eps,
                      bool normalize, const ChainConfig& cfg, int* d_status, cudaStream_t s) {
  ChainParams p{Y, X, G, N, Kp, lo, hi, eps, d_status, cfg.cluster};
  if (hi - lo > cfg.tt || hi - lo > kMaxChainTile) return cudaErrorInvalidValue;
  if (!normalize) return launch_plain(p, s);
  return launch_norm(p, cfg.rpt, s);
}

}  // namespace plnmf
