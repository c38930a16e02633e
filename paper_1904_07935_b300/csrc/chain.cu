// Phase 2 of the regrouped factor update (Alg. 2 inner loop, Eq. 5): the
// columns of one tile are finished one after another.
//
// On entry Y[:, lo:hi] holds, for every row v and column t of the tile,
//   B[v,t] + c'_t X_old[v,t] - sum_{j > t} G[j,t] X_old[v,j]
//                            - sum_{j < lo} G[j,t] X_new[v,j]
// (phase 1 and the phase-3 updates of earlier tiles).  The kernel adds the
// remaining contributions of new columns inside the tile, clamps at eps and,
// for W, divides every finished column by its L2 norm before the next column
// uses it (Alg. 1's W loop).  Each thread keeps its rows' tile of Y in
// registers; when column t is final its value is pushed into the later
// columns of the tile ("right-looking"), so a column costs one clamp, one
// square and the norm reduction on the critical path.
//
// The norm needs every row, so the W chain runs on one thread-block cluster
// (16 CTAs where the GPU allows, else 8): every warp reduces its rows with
// shuffles and sends the partial to every CTA of the cluster with st.async
// into distributed shared memory, completing a transaction count on the
// receiver's mbarrier; every warp waits on its own CTA's mbarrier and adds
// all partials in a fixed order, so all warps (and all runs) see the same
// norm.  Two slot sets alternate between consecutive columns.  Every wait is
// bounded; on expiry the kernel sets ST_TIMEOUT and stops waiting.
//
// The H update (no normalisation, rows independent) uses the same kernel
// without the cluster reduction on a grid covering all rows.
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"

namespace plnmf {
namespace {

struct ChainParams {
  float* Y;
  float* X;
  const float* G;
  int N, Kp, lo, hi;
  int prev_lo;            // >= 0: add the new columns [prev_lo, lo) of X first
  float eps;
  int* status;
  int cl;
};

constexpr int kMaxCluster = 16;
constexpr int kPlainThreads = 256;
constexpr int TT = kMaxChainTile;        // register tile width (columns)

// Output buffer of the finished columns: st[(i * TT + t) * (NT + 1) + r]
// holds column t of thread-row r in row group i.
template <int NT>
__device__ __forceinline__ int st_idx(int i, int t, int r) {
  return (i * TT + t) * (NT + 1) + r;
}

// Warp 0 of every CTA only communicates; the other NT - 32 threads ("row
// threads") each keep RPT rows of the tile in registers, every register index
// static and the column loop a real loop.  Invariant at the top of the
// iteration for column t: slot 1 holds column t with every contribution
// applied; slot s >= 2 holds column t + s - 1 with every contribution except
// that of the previous column t - 1 (value xp).  The iteration
//   1. clamps slot 1 (x) and reduces x^2 over the cluster,
//   2. while warp 0 exchanges the partials, applies xp to the later columns
//      and shifts them down one slot in the same fused multiply-add,
//   3. receives the norm and normalises x,
//   4. applies x to the next column only (slot 1), so that the next clamp can
//      start; x becomes xp.
// The exchange: row warps leave shuffle-reduced partials in shared memory;
// warp 0 adds them, sends the CTA's partial to every CTA of the cluster
// (st.async into distributed shared memory, completing a transaction count
// on the receiver's mbarrier), waits for the CL partials, adds them with a
// fixed shuffle tree (same order in every CTA, so every CTA and every run
// sees the same norm) and publishes 1 / norm.
//
// Rows of CTA `rank`: row group i holds rows rank * NR + i * CL * NR + [0, NR)
// (NR = NT - 32 row threads), i.e. NR consecutive rows; the tile of a row
// group is moved between global memory and the staging buffer with four
// lanes per row (64 contiguous bytes), then between the buffer and registers.
template <int NT, int RPT, bool NORM>
__global__ void __launch_bounds__(NT) chain_kernel(ChainParams p) {
  constexpr int NW = NT / 32;
  constexpr int NR = NT - 32;                    // row threads
  constexpr int NS = TT + 1;                     // register slots per row
  extern __shared__ __align__(16) float st[];    // RPT x TT x (NR + 1)
  __shared__ float Gs[TT][2 * TT];               // G block, zero beyond the tile
  __shared__ __align__(16) float Gp[TT][TT];     // G[prev_lo + j][lo + c] (tail)
  __shared__ float wpart[NW];
  __shared__ float cpart[2][kMaxCluster];
  __shared__ float col_inv;
  __shared__ __align__(8) unsigned long long mbar[2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tr = tid - 32;                       // row-thread index (warps 1..NW-1)
  const int Tw = p.hi - p.lo;
  const unsigned rank = NORM ? cluster_ctarank() : blockIdx.x;
  const int CL = NORM ? p.cl : (int)gridDim.x;
  const int cta_base = (int)rank * NR;
  const int stride = CL * NR;

  for (int e = tid; e < TT * 2 * TT; e += NT) {
    const int i = e / (2 * TT), j = e % (2 * TT);
    Gs[i][j] = (i < Tw && j < Tw) ? p.G[(int64_t)(p.lo + i) * p.Kp + p.lo + j] : 0.f;
  }
  const int Tp = p.prev_lo >= 0 ? p.lo - p.prev_lo : 0;    // width of the previous tile
  for (int e = tid; e < TT * TT; e += NT) {
    const int i = e / TT, j = e % TT;
    Gp[i][j] = (i < Tp && j < Tw) ? p.G[(int64_t)(p.prev_lo + i) * p.Kp + p.lo + j] : 0.f;
  }
  if (NORM && tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    // Expect the first two columns' partials before anyone can send them.
    mbar_arrive_expect_tx(smem_u32(&mbar[0]), CL * 4);
    if (Tw > 1) mbar_arrive_expect_tx(smem_u32(&mbar[1]), CL * 4);
    fence_mbar_init();
  }
  if (NORM) cluster_arrive();                    // the wait comes after the loads

  // Coalesced load of the tile: 4 lanes per row, 16 bytes each; up to four
  // loads per thread are in flight before their shared-memory stores.
  const bool vec = (p.lo & 3) == 0;
  const int total = RPT * NR * 4;
  for (int base = tid; base < total; base += 4 * NT) {
    float v[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * NT;
      const int i = e / (NR * 4), rem = e % (NR * 4);
      const int r = rem >> 2, q = rem & 3;
      const int row = cta_base + i * stride + r;
#pragma unroll
      for (int j = 0; j < 4; ++j) v[u][j] = 0.f;
      if (e < total && row < p.N) {
        const float* src = p.Y + (int64_t)row * p.Kp + p.lo + 4 * q;
        if (vec && 4 * q + 3 < Tw) {
          const float4 f = *reinterpret_cast<const float4*>(src);
          v[u][0] = f.x; v[u][1] = f.y; v[u][2] = f.z; v[u][3] = f.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) v[u][j] = 4 * q + j < Tw ? src[j] : 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * NT;
      if (e >= total) continue;
      const int i = e / (NR * 4), rem = e % (NR * 4);
      const int r = rem >> 2, q = rem & 3;
#pragma unroll
      for (int j = 0; j < 4; ++j) st[(i * TT + 4 * q + j) * (NR + 1) + r] = v[u][j];
    }
  }
  __syncthreads();
  float y[RPT][NS];
  bool valid[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    valid[i] = warp > 0 && cta_base + i * stride + tr < p.N;
    y[i][0] = 0.f;
#pragma unroll
    for (int t = 0; t < TT; ++t) y[i][1 + t] = warp > 0 ? st[(i * TT + t) * (NR + 1) + tr] : 0.f;
  }
  // Contribution of the previous tile's new columns (the base was formed
  // before they were final): y[c] -= sum_j G[prev_lo + j][lo + c] x_new[j].
  // Four columns j at a time: the rows' values as one 16-byte load each, the
  // G block as broadcast 16-byte shared loads reused by every row.
  if (Tp > 0 && warp > 0) {
    const bool pvec = (p.prev_lo & 3) == 0;
#pragma unroll 1
    for (int jq = 0; jq < TT / 4; ++jq) {
      if (4 * jq >= Tp) break;
      float xn[RPT][4];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const float* xr = p.X + (int64_t)(valid[i] ? cta_base + i * stride + tr : 0) * p.Kp + p.prev_lo + 4 * jq;
        if (valid[i] && pvec && 4 * jq + 3 < Tp) {
          const float4 f = *reinterpret_cast<const float4*>(xr);
          xn[i][0] = f.x; xn[i][1] = f.y; xn[i][2] = f.z; xn[i][3] = f.w;
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) xn[i][u] = (valid[i] && 4 * jq + u < Tp) ? xr[u] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int cq = 0; cq < TT / 4; ++cq) {
          const float4 g = *reinterpret_cast<const float4*>(&Gp[4 * jq + u][4 * cq]);
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            y[i][1 + 4 * cq] = fmaf(-g.x, xn[i][u], y[i][1 + 4 * cq]);
            y[i][2 + 4 * cq] = fmaf(-g.y, xn[i][u], y[i][2 + 4 * cq]);
            y[i][3 + 4 * cq] = fmaf(-g.z, xn[i][u], y[i][3 + 4 * cq]);
            y[i][4 + 4 * cq] = fmaf(-g.w, xn[i][u], y[i][4 + 4 * cq]);
          }
        }
      }
    }
  }
  if (NORM) cluster_wait();

  float xp[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) xp[i] = 0.f;
  bool dead = false;
#pragma unroll 1
  for (int t = 0; t < Tw; ++t) {
    float x[RPT];
    const int b = t & 1;
    if (warp > 0) {
      float ss = 0.f;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        x[i] = fmaxf(p.eps, y[i][1]);
        if (valid[i]) ss = fmaf(x[i], x[i], ss);
      }
      if (NORM) {
        ss = warp_sum(ss);
        if (lane == 0) wpart[warp] = ss;
      }
    }
    if (NORM) __syncthreads();
    if (warp > 0) {
      // Step 2: the previous column into the later ones, shifted down a slot.
      if (t > 0) {
#pragma unroll
        for (int s = 2; s < NS; ++s) {
          const float g = Gs[t - 1][t + s - 1];   // slot s holds column t + s - 1
#pragma unroll
          for (int i = 0; i < RPT; ++i) y[i][s - 1] = fmaf(-xp[i], g, y[i][s]);
        }
      } else {
#pragma unroll
        for (int s = 2; s < NS; ++s)
#pragma unroll
          for (int i = 0; i < RPT; ++i) y[i][s - 1] = y[i][s];
      }
    } else if (NORM) {
      float v = (lane >= 1 && lane < NW) ? wpart[lane] : 0.f;
      v = warp_sum(v);
      if (lane < CL && !dead) {
        const unsigned raddr = mapa_u32(smem_u32(&cpart[b][rank]), lane);
        const unsigned rbar = mapa_u32(smem_u32(&mbar[b]), lane);
        st_async_f32(raddr, v, rbar);
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
              if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
              break;
            }
          }
        }
      }
      dead = __any_sync(0xffffffffu, dead);
      // Sum of the CL partials as a fixed shuffle tree.
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
    if (NORM) __syncthreads();
    if (warp > 0) {
      if (NORM) {
        const float inv = col_inv;
#pragma unroll
        for (int i = 0; i < RPT; ++i) x[i] *= inv;
      }
#pragma unroll
      for (int i = 0; i < RPT; ++i) st[(i * TT + t) * (NR + 1) + tr] = x[i];
      // Step 4: the new column into the next one only (critical path).
      const float g1 = Gs[t][t + 1];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        y[i][1] = fmaf(-x[i], g1, y[i][1]);
        xp[i] = x[i];
      }
    }
  }
  __syncthreads();
  // Coalesced store of the finished tile.
  for (int e = tid; e < RPT * NR * 4; e += NT) {
    const int i = e / (NR * 4), rem = e % (NR * 4);
    const int r = rem >> 2, q = rem & 3;
    const int row = cta_base + i * stride + r;
    if (row >= p.N) continue;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = st[(i * TT + 4 * q + j) * (NR + 1) + r];
    float* dst = p.X + (int64_t)row * p.Kp + p.lo + 4 * q;
    if (vec && 4 * q + 3 < Tw) {
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * q + j < Tw) dst[j] = v[j];
    }
  }
  // No CTA may leave while a peer can still write into its shared memory
  // (after a timeout, stores may still be in flight: bounded grace period).
  if (NORM) {
    if (__syncthreads_or(dead ? 1 : 0)) drain_grace();
    cluster_sync_all();
  }
}

size_t chain_smem_bytes(int rpt, int nt) { return sizeof(float) * (size_t)rpt * TT * (nt - 32 + 1); }

template <int NT, int RPT>
cudaError_t launch_norm_t(const ChainParams& p, cudaStream_t s) {
  auto kern = chain_kernel<NT, RPT, true>;
  const size_t smem = chain_smem_bytes(RPT, NT);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.cl > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.cl, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
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

cudaError_t launch_norm(const ChainParams& p, int nt, int rpt, cudaStream_t s) {
  if (nt == 256) {
    switch (rpt) {
      case 1: return launch_norm_t<256, 1>(p, s);
      case 2: return launch_norm_t<256, 2>(p, s);
      case 3: return launch_norm_t<256, 3>(p, s);
      case 4: return launch_norm_t<256, 4>(p, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (nt == 512) {
    switch (rpt) {
      case 1: return launch_norm_t<512, 1>(p, s);
      case 2: return launch_norm_t<512, 2>(p, s);
      case 3: return launch_norm_t<512, 3>(p, s);
      case 4: return launch_norm_t<512, 4>(p, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_plain(const ChainParams& p, cudaStream_t s) {
  const int blocks = std::max(1, (p.N + kPlainThreads - 32 - 1) / (kPlainThreads - 32));
  const size_t smem = chain_smem_bytes(1, kPlainThreads);
  auto kern = chain_kernel<kPlainThreads, 1, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kPlainThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int NT>
int max_cluster_for(int rpt) {
  const size_t smem = chain_smem_bytes(rpt, NT);
  auto kern = chain_kernel<NT, 4, true>;   // the widest variant bounds the others
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int cl : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
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

// Chooses the CTA size, cluster size and rows per thread: at most 4 rows of
// 16 columns in registers per thread; 256-thread CTAs while that suffices,
// else 512-thread CTAs (up to 16 * 480 * 4 = 30,720 rows).
bool chain_config_for(int N, bool normalize, int T, ChainConfig* cfg) {
  if (T < 1 || T > kMaxChainTile) return false;
  if (!normalize) {
    cfg->cluster = 1;
    cfg->threads = kPlainThreads;
    cfg->rpt = 1;
    cfg->tt = T;
    return true;
  }
  for (int nt : {256, 512}) {
    for (int cl : {16, 8}) {
      const int nr = nt - 32;
      const int rpt = (N + cl * nr - 1) / (cl * nr);
      if (rpt > 4) continue;
      const int got = nt == 256 ? max_cluster_for<256>(rpt) : max_cluster_for<512>(rpt);
      if (got < cl) continue;
      cfg->cluster = cl;
      cfg->threads = nt;
      cfg->rpt = rpt;
      cfg->tt = T;
      return true;
    }
  }
  return false;
}

// Same, for a given cluster size (1..16 CTAs): false when the rows do not fit
// 4 per thread or the cluster cannot be resident.
bool chain_config_cluster(int N, int T, int cl, ChainConfig* cfg) {
  if (T < 1 || T > kMaxChainTile || cl < 1 || cl > kMaxCluster) return false;
  for (int nt : {256, 512}) {
    const int nr = nt - 32;
    const int rpt = (N + cl * nr - 1) / (cl * nr);
    if (rpt > 4) continue;
    const int got = nt == 256 ? max_cluster_for<256>(rpt) : max_cluster_for<512>(rpt);
    if (got < cl) continue;
    cfg->cluster = cl;
    cfg->threads = nt;
    cfg->rpt = rpt;
    cfg->tt = T;
    return true;
  }
  return false;
}

cudaError_t chain_run(float* Y, float* X, const float* G, int N, int Kp, int lo, int hi, int prev_lo, float eps,
                      bool normalize, const ChainConfig& cfg, int* d_status, cudaStream_t s) {
  ChainParams p{Y, X, G, N, Kp, lo, hi, prev_lo, eps, d_status, cfg.cluster};
  if (hi - lo > cfg.tt || hi - lo > kMaxChainTile) return cudaErrorInvalidValue;
  if (prev_lo >= 0 && (lo - prev_lo < 1 || lo - prev_lo > kMaxChainTile)) return cudaErrorInvalidValue;
  if (!normalize) return launch_plain(p, s);
  return launch_norm(p, cfg.threads, cfg.rpt, s);
}

}  // namespace plnmf
