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

template <int TT, int RPT, int NT, bool NORM>
__global__ void __launch_bounds__(NT) chain_kernel(ChainParams p) {
  constexpr int NW = NT / 32;
  __shared__ float Gs[TT][TT];
  __shared__ float wpart[NW];
  __shared__ float cpart[2][kMaxCluster];
  __shared__ __align__(8) unsigned long long mbar[2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Tw = p.hi - p.lo;
  const unsigned rank = NORM ? cluster_ctarank() : blockIdx.x;
  const int CL = NORM ? p.cl : (int)gridDim.x;

  for (int e = tid; e < TT * TT; e += NT) {
    const int i = e / TT, j = e % TT;
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
  __syncthreads();
  if (NORM) cluster_sync_all();

  // Rows owned by this thread.
  int row[RPT];
  bool valid[RPT];
  float y[RPT][TT];
  const int base = (int)rank * NT + tid;
  const int stride = CL * NT;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    row[i] = base + i * stride;
    valid[i] = row[i] < p.N;
    const float* src = p.Y + (int64_t)(valid[i] ? row[i] : 0) * p.Kp + p.lo;
#pragma unroll
    for (int t = 0; t < TT; ++t) y[i][t] = (valid[i] && t < Tw) ? src[t] : 0.f;
  }

  bool dead = false;
#pragma unroll
  for (int t = 0; t < TT; ++t) {
    if (t < Tw) {
      float ss = 0.f;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const float v = fmaxf(p.eps, y[i][t]);
        y[i][t] = v;
        if (valid[i]) ss = fmaf(v, v, ss);
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
        }
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
                atomicOr(p.status, ST_TIMEOUT);
                break;
              }
            }
          }
        }
        float tot = 0.f;
        for (int j = 0; j < CL; ++j) tot += cpart[b][j];
        if (tid == 0 && t + 2 < Tw && !dead) mbar_arrive_expect_tx(smem_u32(&mbar[b]), CL * 4);
        const float nrm = sqrtf(tot);
        if (!(nrm > 0.f) || !(nrm < INFINITY)) {
          if (tid == 0 && rank == 0) atomicOr(p.status, ST_NUMERIC);
        }
#pragma unroll
        for (int i = 0; i < RPT; ++i) y[i][t] = y[i][t] / nrm;
      }
      // New column t contributes to the later columns of the tile.
#pragma unroll
      for (int t2 = t + 1; t2 < TT; ++t2) {
        if (t2 < Tw) {
          const float g = Gs[t][t2];
#pragma unroll
          for (int i = 0; i < RPT; ++i) y[i][t2] = fmaf(-y[i][t], g, y[i][t2]);
        }
      }
    }
  }

#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    if (!valid[i]) continue;
    float* dst = p.X + (int64_t)row[i] * p.Kp + p.lo;
#pragma unroll
    for (int t = 0; t < TT; ++t)
      if (t < Tw) dst[t] = y[i][t];
  }
  // No CTA may leave while a peer can still write into its shared memory.
  if (NORM) cluster_sync_all();
}

template <int TT, int RPT, int NT>
cudaError_t launch_norm(const ChainParams& p, cudaStream_t s) {
  auto kern = chain_kernel<TT, RPT, NT, true>;
  if (p.cl > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.cl, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
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

template <int TT, int RPT, int NT>
cudaError_t launch_plain(const ChainParams& p, cudaStream_t s) {
  const int per = NT * RPT;
  const int blocks = std::max(1, (p.N + per - 1) / per);
  chain_kernel<TT, RPT, NT, false><<<blocks, NT, 0, s>>>(p);
  return cudaGetLastError();
}

template <int TT, int RPT, int NT>
int max_cluster_for() {
  auto kern = chain_kernel<TT, RPT, NT, true>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 8;
  }
  for (int cl : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
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

// Chooses the kernel shape: rows per thread and register tile width.
bool chain_config_for(int N, bool normalize, int T, ChainConfig* cfg) {
  if (!normalize) {
    cfg->cluster = 1;
    cfg->threads = 256;
    cfg->rpt = 1;
    cfg->tt = 16;
    return T <= 16;
  }
  int cl = max_cluster_for<16, 2, 1024>();
  if (cl == 0) return false;
  cfg->cluster = cl;
  const long long cap1 = (long long)cl * 1024;
  if (T <= 16 && N <= cap1) { cfg->threads = 1024; cfg->rpt = 1; cfg->tt = 16; return true; }
  if (T <= 16 && N <= 2 * cap1) { cfg->threads = 1024; cfg->rpt = 2; cfg->tt = 16; return true; }
  if (T <= 8 && N <= 4 * cap1) { cfg->threads = 1024; cfg->rpt = 4; cfg->tt = 8; return true; }
  if (T <= 8 && N <= (long long)cl * 512 * 8) { cfg->threads = 512; cfg->rpt = 8; cfg->tt = 8; return true; }
  return false;
}

cudaError_t chain_run(float* Y, float* X, const float* G, int N, int Kp, int lo, int hi, float eps,
                      bool normalize, const ChainConfig& cfg, int* d_status, cudaStream_t s) {
  ChainParams p{Y, X, G, N, Kp, lo, hi, eps, d_status, cfg.cluster};
  if (!normalize) return launch_plain<16, 1, 256>(p, s);
  if (cfg.tt == 16 && cfg.rpt == 1) return launch_norm<16, 1, 1024>(p, s);
  if (cfg.tt == 16 && cfg.rpt == 2) return launch_norm<16, 2, 1024>(p, s);
  if (cfg.tt == 8 && cfg.rpt == 4) return launch_norm<8, 4, 1024>(p, s);
  if (cfg.tt == 8 && cfg.rpt == 8) return launch_norm<8, 8, 512>(p, s);
  return cudaErrorInvalidConfiguration;
}

}  // namespace plnmf
