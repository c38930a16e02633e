// The whole W update (Alg. 1's W loop in the tiled order of Alg. 2) as
// one persistent launch.
//
// W is updated in tiles of 16 columns.  Column t of tile [lo, hi) is
//   w_t = max(eps, P_t - sum_{j < t} Q[j][t] w_j(new) - sum_{j > t} Q[j][t] w_j(old)),
// then divided by its L2 norm before any later column uses it.  (Alg. 2's
// W_old * Q_tt initialisation cancels the j = t term of Eq. 5 exactly and is
// left out.)
//
// Two grids run side by side: the chain grid (one cluster of CL = 16 CTAs,
// whose CTAs the hardware runs together) and the worker grid (one CTA per
// remaining SM, no clusters, so every SM outside the chain's cluster takes
// a share of the bases; a single launch would need clusters of 16 for the
// workers too, and only 7 such clusters fit on the 148 SMs).  The worker
// grid is launched after the chain grid as a programmatic dependent: it may
// start once every chain CTA is running, and nothing below assumes that it
// runs at the same time as the chain, or at all:
// Hand-off through global memory.  The rows are cut into nb blocks (one per
// worker CTA); block (tau, w) of a tile base is computed by whoever claims
// it first (atomic compare-and-swap on its state word): normally worker w,
// which claims it as soon as the chain has published tile tau - 2
// (chain_done[tau]); when the chain reaches tile tau it claims every block
// still unclaimed and computes it itself, with the same arithmetic in the
// same order.  base_done[tau] counts finished blocks.  So the chain only ever
// waits for blocks claimed by a CTA that is running and needs nothing more to
// finish them, and a worker that finds the chain not yet running leaves its
// remaining blocks to it: the update completes whatever subset of the
// worker CTAs is resident at a time.  The worker grid ends only after the
// chain has finished (a release count of the chain CTAs that every worker
// CTA waits for), so work ordered after the two launches sees the whole
// update.  Release/acquire ordering, and every wait is bounded by the global
// timer (ST_TIMEOUT on expiry).
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"
#include "tcutil.cuh"

namespace plnmf {
namespace {

constexpr int WT = kRowTile;        // tile width (16)
constexpr int WNT = 512;            // threads per CTA
constexpr int WNR = WNT - 32;       // row threads of a chain CTA
constexpr int WMAXCL = 16;
constexpr int WMAXNB = 160;         // blocks per tile (worker CTAs: one per SM outside the chain)

struct WParams {
  float* X;            // N x Kp, old on entry, new on exit
  const float* P;      // N x Kp
  const float* Q;      // Kp x Kp
  int N, K, Kp;
  float eps;
  int* status;
  int* sync;           // hand-off words, w_sync_ints(K) ints (layout: sync_* below)
  int cl;              // CTAs per cluster (chain cluster size)
  int worker_rows;     // rows per worker pass (4 lanes per row)
  int chain_rows;      // rows per chain CTA, ceil(N / cl): CTA rank owns [rank * chain_rows, ...)
  int nb;              // row blocks per tile base: block w = rows [w * per, min(N, (w + 1) * per))
  int per;
  const float* pre0;   // non-null: Yc's slot 0 + pre0 (the same order) hold tile 0's base less P (formed before the launch)
  unsigned long long wait_ns;  // limit of every wait
  int extra_arrivals;  // added to the chain_done count the workers wait for (tests of the timeout path; 0)
  float* spart;        // non-null: chunk w (w < nb) of the Gram partials S_w = X_w^T X_w of the new factor,
                       // Kp x Kp each, upper triangle (the rows of worker w are the chunk)
  int stage_rows;      // rows a worker stages at once (>= worker_rows; per: its whole block)
  float* Yc;           // tile bases in the chain's register order (yc_quad), two tile slots
  int rpt;             // register rows per chain row thread
};

__device__ __forceinline__ unsigned cluster_id_x() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}

// Hand-off counters live one per 128-byte line (kSyncStride ints apart), so
// the workers' polling and the chain's release do not share a line:
// counter 0 counts the chain CTAs that started, counters 1 .. nt the chain
// CTAs that stored tile tau (chain_done), counters nt + 1 .. 2 nt the finished blocks
// of tile tau's base (base_done); then nt x WMAXNB block states (0 free,
// 1 claimed).
constexpr int kSyncStride = 32;
__device__ __forceinline__ int* sync_started(const WParams& p) { return p.sync; }
__device__ __forceinline__ int* sync_chain_done(const WParams& p, int nt, int tau) {
  return p.sync + (1 + tau) * kSyncStride;
}
__device__ __forceinline__ int* sync_base_done(const WParams& p, int nt, int tau) {
  return p.sync + (1 + nt + tau) * kSyncStride;
}
__device__ __forceinline__ int* sync_state(const WParams& p, int nt, int tau, int w) {
  return p.sync + (1 + 2 * nt) * kSyncStride + tau * WMAXNB + w;
}
// Block columns of the Gram partials finished by the workers (nb x nt when
// complete).
__device__ __forceinline__ int* sync_sdone(const WParams& p, int nt) {
  return p.sync + (1 + 2 * nt) * kSyncStride + nt * WMAXNB;
}
// Chain CTAs that have finished (every store released).
__device__ __forceinline__ int* sync_finished(const WParams& p, int nt) {
  return p.sync + (2 + 2 * nt) * kSyncStride + nt * WMAXNB;
}

// Tile bases in the order the chain's row threads hold them: tile tau in
// slot tau & 1; in a slot, chain CTA c, register row i, column quad q and
// row thread r give the 16-byte quad of row c * chain_rows + i * WNR + r,
// columns 4 q .. 4 q + 3 of the tile (zero past K).  A row thread loads its
// whole tile with RPT x 4 loads, each a warp's 512 consecutive bytes.  Two
// slots suffice: the base of tile tau is written only after every chain CTA
// has published tile tau - 2, so after it has loaded the base of tile
// tau - 2 (the chain's own blocks of tile tau are formed at tile tau).
static_assert(WNR == kChainRowThreads, "chain register order");
__device__ __forceinline__ float4* yc_quad(const WParams& p, int tau, int v, int q) {
  return reinterpret_cast<float4*>(p.Yc) + (int64_t)(tau & 1) * p.cl * p.rpt * 4 * WNR +
         chain_quad(v, q, p.chain_rows, p.rpt);
}

// A worker that finds the chain cluster not yet running waits this long for
// it before leaving its remaining blocks to the chain.
constexpr unsigned long long kGiveUpNs = 50ull * 1000ull;

// Bounded spin with exponential backoff (32 ns .. 512 ns between polls, so
// that many waiting CTAs do not keep the line's L2 slice busy) until *p >=
// target.  Returns 1 when reached, 0 when the wait ran out (ST_TIMEOUT set),
// 2 when `started` (if given) showed fewer than `need` CTAs after kGiveUpNs
// (no error: the caller leaves the work to those CTAs).
__device__ int wait_count(const int* p, int target, const WParams& prm, const int* started = nullptr,
                          int need = 0) {
  unsigned long long t0 = 0;
  unsigned polls = 0;
  unsigned sleep_ns = 32;
  while (ld_acquire_gpu(p) < target) {
    __nanosleep(sleep_ns);
    if (sleep_ns < 512) sleep_ns <<= 1;
    if ((++polls & 15u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) {
        t0 = now;
      } else {
        const unsigned long long el = now - t0;
        if (started && el > kGiveUpNs && ld_acquire_gpu(started) < need) return 2;
        if (el > prm.wait_ns) {
          atomicOr(prm.status, ST_TIMEOUT);
          return 0;
        }
      }
    }
  }
  return 1;
}

// Bounded wait for the phase `parity` of a CTA-local mbarrier (bulk copies).
__device__ bool wait_bar_cta(unsigned bar, unsigned parity, unsigned long long limit) {
  unsigned long long t0 = 0;
  unsigned polls = 0;
  while (!mbar_try_wait_cta(bar, parity)) {
    if ((++polls & 63u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit) return false;
    }
  }
  return true;
}

// Bounded wait for the phase `parity` of a CTA's mbarrier that remote CTAs
// of the cluster complete (the column partials).
__device__ bool wait_bar_cluster(unsigned bar, unsigned parity, unsigned long long limit) {
  unsigned long long t0 = 0;
  unsigned polls = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++polls & 31u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit) return false;
    }
  }
  return true;
}

// --------------------------------------------------------------------------
// One row of a tile base from global memory (the chain's path for blocks no
// worker claimed).  The operations and their order are those of the worker
// below (Gc[j][c] = Q[j][lo + c], zero past K; blocks of WT terms folded with
// comp_fold; the in-tile old terms last), so either path gives the same bits.
// --------------------------------------------------------------------------
__device__ __forceinline__ void base_row_global(const WParams& p, int v, int lo, int hi, int new_end) {
  const float* xr = p.X + (int64_t)v * p.Kp;
  auto gq = [&](int j, int c) -> float {
    return (j < p.K && lo + c < p.K) ? __ldg(p.Q + (int64_t)j * p.Kp + lo + c) : 0.f;
  };
  float acc[WT], cmp[WT], blk[WT];
#pragma unroll
  for (int c = 0; c < WT; ++c) {
    acc[c] = lo + c < hi ? __ldg(p.P + (int64_t)v * p.Kp + lo + c) : 0.f;
    cmp[c] = blk[c] = 0.f;
  }
  auto step = [&](int j) {
    const float4 x4 = *reinterpret_cast<const float4*>(xr + j);
    const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < WT; ++c) blk[c] = fmaf(gq(j + u, c), xs[u], blk[c]);
  };
  auto fold = [&]() {
#pragma unroll
    for (int c = 0; c < WT; ++c) comp_fold(acc[c], cmp[c], blk[c]);
  };
  auto outside = [&](int j0, int j1) {
    int jb = j0;
#pragma unroll 1
    for (; jb + WT <= j1; jb += WT) {
#pragma unroll 1
      for (int jj = 0; jj < WT; jj += 4) step(jb + jj);
      fold();
    }
    if (jb < j1) {
#pragma unroll 1
      for (int j = jb; j < j1; j += 4) step(j);
      fold();
    }
  };
  outside(0, new_end);
  outside(lo + WT < p.Kp ? lo + WT : p.Kp, p.Kp);
  float xo[WT];
#pragma unroll
  for (int q = 0; q < WT / 4; ++q) {
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lo + 4 * q < p.Kp) t = *reinterpret_cast<const float4*>(xr + lo + 4 * q);
    xo[4 * q] = t.x; xo[4 * q + 1] = t.y; xo[4 * q + 2] = t.z; xo[4 * q + 3] = t.w;
  }
#pragma unroll
  for (int c = 0; c < WT; ++c) acc[c] += cmp[c];
#pragma unroll
  for (int j = 1; j < WT; ++j) {
#pragma unroll
    for (int c = 0; c < WT; ++c)
      if (j > c) acc[c] = fmaf(-gq(lo + j, c), xo[j], acc[c]);
  }
  // (acc is zero past K: so are P's term and every Q factor there.)
#pragma unroll
  for (int q = 0; q < WT / 4; ++q)
    *yc_quad(p, lo / WT, v, q) = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
}

// --------------------------------------------------------------------------
// Worker role: tile bases.
// --------------------------------------------------------------------------
// WR rows per lane group: group g takes rows g and (WR = 2) g + RB / 2 of
// the pass, so that one 16-byte load of Q's block serves WR rows (Kp >= 128,
// where the shared-memory loads bound the workers: text-like K = 160 W update
// 198 -> 194 us; neutral at K = 80); each row's arithmetic is the same
// either way.
template <int WR>
__device__ void worker_role(const WParams& p, char* smem, int wid) {
  const int nt = (p.K + WT - 1) / WT;
  const int Kr = (p.Kp + WT - 1) / WT * WT;
  const int ldx = p.Kp + 4;
  float* Gc = reinterpret_cast<float*>(smem);                 // Kr x WT
  float* Xs = Gc + Kr * WT;                                   // worker_rows x ldx
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int s_go[2];
  const int tid = threadIdx.x;
  const int sub = tid & 3;
  const int rl = tid >> 2;
  const int RB = p.worker_rows;
  const int SR = p.stage_rows;
  const bool s_after = SR >= p.per;                           // the whole block staged at once
  // This worker's block: an equal contiguous share [wbeg, wend) of the rows,
  // in passes of RB rows (rather than RB-row blocks dealt round-robin, which
  // left some workers a whole block more than others: text-like K = 240 W
  // update 513 -> 421 us, K = 320 868 -> 688 us).
  if (wid >= p.nb) return;                                    // no rows (small N)
  const int wbeg = wid * p.per, wend = min(p.N, wbeg + p.per);
  if (tid == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned phase = 0;
  // Rows [row0, row0 + nrows) of the factor into Xs (one bulk copy per row),
  // bounded wait; on expiry the copies may still be in flight, so wait for
  // them once more (bounded too) before the buffer is used or left.
  auto stage_pass = [&](int row0, int nrows) {
    __syncthreads();                                          // Xs free
    if (tid == 0) mbar_arrive_expect_tx(smem_u32(&bar), (unsigned)nrows * p.Kp * 4u);
    __syncthreads();
    if (tid < nrows) {
      fence_proxy_async_global();
      bulk_g2s(smem_u32(Xs + tid * ldx), p.X + (int64_t)(row0 + tid) * p.Kp, (unsigned)p.Kp * 4u, smem_u32(&bar));
    }
    if (!wait_bar_cta(smem_u32(&bar), phase, p.wait_ns)) {
      if (tid == 0) atomicOr(p.status, ST_TIMEOUT);
      wait_bar_cta(smem_u32(&bar), phase, p.wait_ns);
    }
    phase ^= 1u;
  };
  // Gram partial of this worker's rows (WParams::spart), block column sc:
  // entries (i, j), j in [16 sc, 16 sc + 16), i <= j, as 4 x 4 tiles
  // (s_st = tile); each tile has two threads in the two half-warps of one
  // warp, the first taking the 8-row groups 0, 2, 4, ... of the chunk and the
  // second 1, 3, 5, ..., each adding its rows in order (the chunk's rows are
  // final in every column up to the block column once chain_done[sc] is
  // seen); the two sums are then added, the first's plus the second's.  This
  // is the order of gram_tri_kernel's chunk partials, so with the same chunks
  // the two agree bit for bit and either can stand for the other.
  const int s_h = (tid >> 4) & 1;
  const int s_st = (tid & 15) + 16 * (tid >> 5);
  float sacc[4][4];
  auto s_tile = [&](int sc, int* i0, int* j0) -> bool {
    const int slo = sc * WT, shi = min(p.K, slo + WT);
    const int nj = (min(p.Kp, slo + WT) - slo) / 4, niq = (shi + 3) / 4;
    if (s_st >= niq * nj) return false;
    *i0 = 4 * (s_st / nj);
    *j0 = slo + 4 * (s_st % nj);
    return *i0 <= *j0 + 3;                                    // not entirely below the diagonal
  };
  auto s_begin = [&]() {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) sacc[u][v] = 0.f;
  };
  // One row's products into the tile: two columns per instruction (packed
  // FP32 multiply-add, each half rounded as a scalar fmaf).
  auto s_acc = [&](const float4& a4, const float4& b4) {
    const float a[4] = {a4.x, a4.y, a4.z, a4.w};
    const float2 b01 = make_float2(b4.x, b4.y), b23 = make_float2(b4.z, b4.w);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 aa = make_float2(a[u], a[u]);
      float2 l = make_float2(sacc[u][0], sacc[u][1]), r = make_float2(sacc[u][2], sacc[u][3]);
      l = __ffma2_rn(aa, b01, l);
      r = __ffma2_rn(aa, b23, r);
      sacc[u][0] = l.x;
      sacc[u][1] = l.y;
      sacc[u][2] = r.x;
      sacc[u][3] = r.y;
    }
  };
  auto s_rows = [&](int sc, int row0, int nrows) {
    int i0, j0;
    if (!s_tile(sc, &i0, &j0)) return;
    // This half's rows in order: groups g0, g0 + 2, ... of 8 rows; full
    // groups with all eight rows' operands loaded first.
    for (int g = (((row0 - wbeg) >> 3) ^ s_h) & 1; 8 * g < nrows; g += 2) {
      const float* xr = Xs + 8 * g * ldx;
      if (8 * g + 8 <= nrows) {
        float4 a4[8], b4[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          a4[q] = *reinterpret_cast<const float4*>(xr + q * ldx + i0);
          b4[q] = *reinterpret_cast<const float4*>(xr + q * ldx + j0);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) s_acc(a4[q], b4[q]);
      } else {
        for (int q = 0; 8 * g + q < nrows; ++q) {
          const float4 a4 = *reinterpret_cast<const float4*>(xr + q * ldx + i0);
          const float4 b4 = *reinterpret_cast<const float4*>(xr + q * ldx + j0);
          s_acc(a4, b4);
        }
      }
    }
  };
  auto s_finish = [&](int sc) {
    int i0 = 0, j0 = 0;
    const bool own = s_tile(sc, &i0, &j0);                    // the same for both half-warps of a tile
    float* out = p.spart + (int64_t)wid * p.Kp * p.Kp;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float o = __shfl_xor_sync(0xffffffffu, sacc[u][v], 16);
        const int i = i0 + u, j = j0 + v;
        if (own && s_h == 0 && i <= j && j < p.K) out[(int64_t)i * p.Kp + j] = sacc[u][v] + o;
      }
    __syncthreads();                                          // the block column's partial is written
    if (tid == 0) atomicAdd(sync_sdone(p, nt), 1);
  };
  // Columns [c0, c1) of the staged rows from the factor in global memory (the
  // rest of each row is staged already): the last block columns need only
  // their own tiles again.
  auto reload_cols = [&](int c0, int c1) {
    __syncthreads();
    const int q4 = (c1 - c0) / 4, n = wend - wbeg;
    for (int e = tid; e < n * q4; e += WNT) {
      const int r = e / q4, q = e % q4;
      *reinterpret_cast<float4*>(Xs + r * ldx + c0 + 4 * q) =
          __ldcg(reinterpret_cast<const float4*>(p.X + (int64_t)(wbeg + r) * p.Kp + c0 + 4 * q));
    }
    __syncthreads();
  };
  // Tiles [0, xs_final) of the staged rows are final (whole-block staging).
  int xs_final = -1;
  bool gave_up = false;
  for (int tau = 0; tau < nt; ++tau) {
    if (tau == 0 && p.pre0) continue;                         // tile 0's base was formed before the launch
    const int lo = tau * WT, hi = min(p.K, lo + WT);
    const int new_end = tau >= 1 ? lo - WT : 0;
    // go: 1 = this worker computes block (tau, wid); 2 = the chain claimed
    // it; 0 = leave this and every later block to the chain.
    if (tid == 0) {
      int go = 1;
      if (tau >= 2)
        go = wait_count(sync_chain_done(p, nt, tau - 2), p.cl + p.extra_arrivals, p, sync_started(p), p.cl) == 1;
      if (go) go = atomicCAS(sync_state(p, nt, tau, wid), 0, 1) == 0 ? 1 : 2;
      fence_proxy_async_global();
      s_go[tau & 1] = go;
    }
    __syncthreads();
    const int go = s_go[tau & 1];
    if (go == 0) {
      gave_up = true;
      break;
    }
    if (go == 2) continue;
    // Block column tau - 2 of the Gram partial rides on this tile's passes
    // (its columns are final: chain_done[tau - 2] was seen above).
    const int scol = p.spart && tau >= 2 ? tau - 2 : -1;
    if (scol >= 0) s_begin();
    // G block of this tile: Gc[j * WT + c] = Q[j][lo + c].
    for (int base = tid; base < Kr * WT; base += 8 * WNT) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = base + u * WNT;
        const int j = e / WT, c = e % WT;
        v[u] = (e < Kr * WT && j < p.K && lo + c < p.K) ? __ldg(p.Q + (int64_t)j * p.Kp + lo + c) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = base + u * WNT;
        if (e < Kr * WT) Gc[e] = v[u];
      }
    }
    // Rows staged stage_rows at a time (normally the whole block, which
    // then stays in shared memory for the Gram partial below and for the
    // next tiles), the base formed in passes of RB rows over them.
    for (int srow0 = wbeg; srow0 < wend; srow0 += SR) {
     const int snrows = min(SR, wend - srow0);
     if (s_after && xs_final >= 0) {
       // The whole block is staged with tiles [0, xs_final) final and the
       // others old, which is what they still are in global memory: only the
       // tiles finished since (normally tile tau - 2) are fetched again.
       if (xs_final < tau - 1) reload_cols(xs_final * WT, (tau - 1) * WT);
       else __syncthreads();                                  // (after Gc is staged)
       xs_final = max(xs_final, tau - 1);
     } else {
       stage_pass(srow0, snrows);                             // (after Gc is staged)
       xs_final = s_after ? max(0, tau - 1) : -1;
     }
     for (int prow = 0; prow < snrows; prow += RB) {
      const int nrows = min(RB, snrows - prow);
      const int row0 = srow0 + prow;
      const float* Xq = Xs + prow * ldx;
      const int half = WR == 1 ? nrows : (nrows + 1) / 2;  // groups with a row
      if (rl < half) {
        int lr[WR];
        bool has[WR];
        const float* xr[WR];
#pragma unroll
        for (int u = 0; u < WR; ++u) {
          lr[u] = rl + u * half;
          has[u] = lr[u] < nrows;
          xr[u] = Xq + (has[u] ? lr[u] : rl) * ldx;
        }
        float acc[WR][4];
#pragma unroll
        for (int u = 0; u < WR; ++u)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = lo + 4 * sub + q;
            acc[u][q] = (has[u] && c < hi) ? __ldg(p.P + (int64_t)(row0 + lr[u]) * p.Kp + c) : 0.f;
          }
        // Blocks of WT terms folded into acc with compensation (comp_fold).
        float cmp[WR][4], blk[WR][4];
#pragma unroll
        for (int u = 0; u < WR; ++u)
#pragma unroll
          for (int q = 0; q < 4; ++q) cmp[u][q] = blk[u][q] = 0.f;
        auto step = [&](int j) {
          float xs[WR][4];
#pragma unroll
          for (int u = 0; u < WR; ++u) {
            const float4 x4 = *reinterpret_cast<const float4*>(xr[u] + j);
            xs[u][0] = x4.x; xs[u][1] = x4.y; xs[u][2] = x4.z; xs[u][3] = x4.w;
          }
          // Two columns per instruction (packed FP32 multiply-add).
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float4 g = *reinterpret_cast<const float4*>(Gc + (j + v) * WT + 4 * sub);
            const float2 g01 = make_float2(g.x, g.y), g23 = make_float2(g.z, g.w);
#pragma unroll
            for (int u = 0; u < WR; ++u) {
              const float2 xx = make_float2(xs[u][v], xs[u][v]);
              float2 l = make_float2(blk[u][0], blk[u][1]), r = make_float2(blk[u][2], blk[u][3]);
              l = __ffma2_rn(g01, xx, l);
              r = __ffma2_rn(g23, xx, r);
              blk[u][0] = l.x;
              blk[u][1] = l.y;
              blk[u][2] = r.x;
              blk[u][3] = r.y;
            }
          }
        };
        auto fold = [&]() {
#pragma unroll
          for (int u = 0; u < WR; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) comp_fold(acc[u][q], cmp[u][q], blk[u][q]);
        };
        // Full blocks unrolled; a ragged last block step by step.
        auto outside = [&](int j0, int j1) {
          int jb = j0;
#pragma unroll 1
          for (; jb + WT <= j1; jb += WT) {
#pragma unroll
            for (int jj = 0; jj < WT; jj += 4) step(jb + jj);
            fold();
          }
          if (jb < j1) {
#pragma unroll 1
            for (int j = jb; j < j1; j += 4) step(j);
            fold();
          }
        };
        outside(0, new_end);
        outside(lo + WT < p.Kp ? lo + WT : p.Kp, p.Kp);
#pragma unroll
        for (int u = 0; u < WR; ++u) {
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[u][q] += cmp[u][q];
          float xo[WT];
#pragma unroll
          for (int q = 0; q < WT / 4; ++q) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (lo + 4 * q < p.Kp) v = *reinterpret_cast<const float4*>(xr[u] + lo + 4 * q);
            xo[4 * q] = v.x; xo[4 * q + 1] = v.y; xo[4 * q + 2] = v.z; xo[4 * q + 3] = v.w;
          }
#pragma unroll
          for (int j = 1; j < WT; ++j) {
            const float4 g4 = *reinterpret_cast<const float4*>(Gc + (lo + j) * WT + 4 * sub);
            const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int cl = 4 * sub + q;
              if (j > cl) acc[u][q] = fmaf(-gv[q], xo[j], acc[u][q]);
            }
          }
          if (!has[u]) continue;
          // (Zero past K: so are P's term and every Q factor there.)
          *yc_quad(p, tau, row0 + lr[u], sub) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
        }
      }
     }
     if (scol >= 0 && !s_after) s_rows(scol, srow0, snrows);   // block larger than one staging
    }
    // A claimed block is always published (even after a timed-out copy), so
    // the chain never waits for it in vain.
    __syncthreads();
    if (tid == 0) red_release_add_gpu(sync_base_done(p, nt, tau), 1);
    // The Gram partial's block column from the rows still staged: after the
    // base is published, so the chain does not wait for it.
    if (scol >= 0) {
      if (s_after) s_rows(scol, wbeg, wend - wbeg);
      s_finish(scol);
    }
  }
  // The last block columns of the Gram partial (those no later tile's passes
  // carried), each once its tile is final; a worker that gave up, or whose
  // wait runs out here, leaves its remaining columns to the Gram kernel that
  // follows the launch (the completion count falls short).
  if (p.spart && !gave_up) {
    for (int sc = nt >= 2 ? nt - 2 : 0; sc < nt; ++sc) {
      if (tid == 0) {
        const int ok =
            wait_count(sync_chain_done(p, nt, sc), p.cl + p.extra_arrivals, p, sync_started(p), p.cl) == 1;
        fence_proxy_async_global();
        s_go[sc & 1] = ok;
      }
      __syncthreads();
      if (!s_go[sc & 1]) break;
      s_begin();
      if (s_after && xs_final >= 0 && xs_final <= sc) {
        // The block is staged with tiles [0, xs_final) final: fetch tiles
        // xs_final .. sc again.
        reload_cols(xs_final * WT, min(p.Kp, (sc + 1) * WT));
        xs_final = sc + 1;
        s_rows(sc, wbeg, wend - wbeg);
      } else {
        for (int row0 = wbeg; row0 < wend; row0 += SR) {
          const int nrows = min(SR, wend - row0);
          stage_pass(row0, nrows);
          s_rows(sc, row0, nrows);
        }
        xs_final = s_after ? sc + 1 : -1;
      }
      s_finish(sc);
    }
  }
}

// --------------------------------------------------------------------------
// Worker role on the tensor cores: the same tile bases with the off-tile sums
// (Eqs. 4 and 6) as a [128 rows x Kp] x [Kp x 16] product on tcgen05.  The
// operands are split into TF32 pairs (hi = tf32(x), lo = tf32(x - hi); three
// kind::tf32 MMAs per K step, about 2^-21 relative per product); each
// 32-column plane of the rows accumulates in its own 16-column slice of
// tensor memory and the slices are folded into the running value with
// compensation, plane by plane.  The B operand of tile tau is Q[lo + c][j]
// for the columns the base needs (new j < lo - 16, old j >= lo + 16), zero
// elsewhere.  Roles: warps 0-3 one row each (split, fold, epilogue); thread
// 128 streams the planes of 128-row passes (TMA, 128-byte swizzle); thread
// 160 issues the MMAs into one of two halves of tensor memory (pass parity);
// every thread builds B at the start of a tile.
// --------------------------------------------------------------------------
constexpr int WPW = 32;               // FP32 columns per plane
constexpr int WTM = 128;              // rows per pass (TMEM lanes)
constexpr int WPLANE = WTM * 128;     // 16 KB
constexpr int WBPLANE = WT * 128;     // 2 KB
constexpr int WNSMAX = 6;

__host__ __device__ constexpr int wtc_planes(int Kp) { return (Kp + WPW - 1) / WPW; }
__host__ __device__ constexpr int wtc_slots(int Kp) {
  return (200 * 1024 - 4 * wtc_planes(Kp) * WBPLANE) / (2 * WPLANE) > WNSMAX
             ? WNSMAX
             : ((200 * 1024 - 4 * wtc_planes(Kp) * WBPLANE) / (2 * WPLANE) < 2
                    ? 2
                    : (200 * 1024 - 4 * wtc_planes(Kp) * WBPLANE) / (2 * WPLANE));
}
__host__ __device__ constexpr unsigned wtc_tmem_cols(int Kp) {
  return 2 * wtc_planes(Kp) * WT <= 32    ? 32u
         : 2 * wtc_planes(Kp) * WT <= 64  ? 64u
         : 2 * wtc_planes(Kp) * WT <= 128 ? 128u
         : 2 * wtc_planes(Kp) * WT <= 256 ? 256u
                                           : 512u;
}
size_t wtc_smem(int Kp) {
  return (size_t)2 * wtc_slots(Kp) * WPLANE + (size_t)2 * wtc_planes(Kp) * WBPLANE + 1024;
}

__device__ void worker_role_tc(const WParams& p, char* smem_raw, int wid, const CUtensorMap* mapX) {
  if (wid >= p.nb) return;                                    // no rows (small N)
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nt = (p.K + WT - 1) / WT;
  const int P = wtc_planes(p.Kp), NS = wtc_slots(p.Kp);
  const unsigned cols = wtc_tmem_cols(p.Kp);
  char* ahi = smem;
  char* alo = smem + NS * WPLANE;
  char* bhi = smem + 2 * NS * WPLANE;
  char* blo = bhi + P * WBPLANE;
  __shared__ __align__(8) unsigned long long full[WNSMAX], loready[WNSMAX], empty[WNSMAX];
  __shared__ __align__(8) unsigned long long done[2], tfree[2], fin;
  __shared__ unsigned tmem_slot;
  __shared__ int s_go[2];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wbeg = wid * p.per, wend = min(p.N, wbeg + p.per);
  const int npass = (wend - wbeg + WTM - 1) / WTM;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&loready[s]), WTM);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(smem_u32(&done[h]), 1);
      mbar_init(smem_u32(&tfree[h]), WTM);
    }
    mbar_init(smem_u32(&fin), 1);
    fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const unsigned tmem = tmem_slot;
  bool dead = false;
  auto bwait = [&](unsigned long long* bar, unsigned parity) {
    if (dead) return;
    if (!tc::wait(smem_u32(bar), parity, p.wait_ns)) {
      atomicOr(p.status, ST_TIMEOUT);
      dead = true;
    }
  };
  int gp = 0, gc = 0;                                         // passes / planes streamed so far
  int issued[WNSMAX] = {0, 0, 0, 0, 0, 0};
  for (int tau = 0; tau < nt; ++tau) {
    if (tau == 0 && p.pre0) continue;                         // tile 0's base was formed before the launch
    const int lo = tau * WT, hi = min(p.K, lo + WT), w = hi - lo;
    const int new_end = tau >= 1 ? lo - WT : 0;
    if (tid == 0) {
      int go = 1;
      if (tau >= 2)
        go = wait_count(sync_chain_done(p, nt, tau - 2), p.cl + p.extra_arrivals, p, sync_started(p), p.cl) == 1;
      if (go) go = atomicCAS(sync_state(p, nt, tau, wid), 0, 1) == 0 ? 1 : 2;
      fence_proxy_async_global();
      s_go[tau & 1] = go;
    }
    __syncthreads();
    const int go = s_go[tau & 1];
    if (go == 0) break;
    if (go == 2) continue;
    // B operand of this tile (every thread; the previous tile's MMAs are
    // complete: its last pass was read before the barrier above).
    for (int e = tid; e < WT * P * WPW; e += WNT) {
      const int c = e / (P * WPW), j = e % (P * WPW);
      const bool in = j < p.K && lo + c < p.K && (j < new_end || j >= lo + WT);
      const float v = in ? __ldg(p.Q + (int64_t)(lo + c) * p.Kp + j) : 0.f;
      const float h = tc::tf32_rn(v), l = tc::tf32_rn(v - h);
      const unsigned off = (unsigned)((j / WPW) * WBPLANE) + tc::sw128_off(c, (j % WPW) * 4);
      *reinterpret_cast<float*>(bhi + off) = h;
      *reinterpret_cast<float*>(blo + off) = l;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid < WTM) {
      // ---- rows: split the planes, fold the slices, form and store the base
      const unsigned lane_base = (unsigned)(warp * 32) << 16;
      for (int k = 0; k < npass; ++k) {
        const int gpk = gp + k, half = gpk & 1;
        for (int q = 0; q < P; ++q) {
          const int g = gc + k * P + q, s = g % NS;
          bwait(&full[s], (unsigned)(g / NS) & 1u);
          char* ph = ahi + s * WPLANE;
          char* pl = alo + s * WPLANE;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const unsigned off = tc::sw128_off(tid, u * 16);
            const float4 v = *reinterpret_cast<const float4*>(ph + off);
            float4 h4, l4;
            h4.x = tc::tf32_rn(v.x); l4.x = tc::tf32_rn(v.x - h4.x);
            h4.y = tc::tf32_rn(v.y); l4.y = tc::tf32_rn(v.y - h4.y);
            h4.z = tc::tf32_rn(v.z); l4.z = tc::tf32_rn(v.z - h4.z);
            h4.w = tc::tf32_rn(v.w); l4.w = tc::tf32_rn(v.w - h4.w);
            *reinterpret_cast<float4*>(ph + off) = h4;
            *reinterpret_cast<float4*>(pl + off) = l4;
          }
          tc::fence_async_smem();
          mbar_arrive(smem_u32(&loready[s]));
        }
        const int v = wbeg + k * WTM + tid;
        const bool valid = v < wend;
        float acc[WT], cmp[WT];
#pragma unroll
        for (int c = 0; c < WT; ++c) {
          acc[c] = valid && c < w ? __ldg(p.P + (int64_t)v * p.Kp + lo + c) : 0.f;
          cmp[c] = 0.f;
        }
        bwait(&done[half], (unsigned)(gpk >> 1) & 1u);
        tc::fence_after();
        for (int q = 0; q < P; ++q) {
          float blk[WT];
          tc::tmem_ld16(tmem + lane_base + (unsigned)((half * P + q) * WT), blk);
#pragma unroll
          for (int c = 0; c < WT; ++c) comp_fold(acc[c], cmp[c], blk[c]);
        }
        tc::fence_before();
        mbar_arrive(smem_u32(&tfree[half]));
#pragma unroll
        for (int c = 0; c < WT; ++c) acc[c] += cmp[c];
        if (valid) {
          // Old in-tile columns j > c.
          const float* xr = p.X + (int64_t)v * p.Kp + lo;
          float xo[WT];
#pragma unroll
          for (int c = 0; c < WT; ++c) xo[c] = c < w ? xr[c] : 0.f;
          const float* gt = p.Q + (int64_t)lo * p.Kp + lo;
#pragma unroll
          for (int j = 1; j < WT; ++j)
#pragma unroll
            for (int c = 0; c < WT; ++c)
              if (j > c && j < w) acc[c] = fmaf(-__ldg(gt + (int64_t)j * p.Kp + c), xo[j], acc[c]);
          // (Zero past K: so are P's term, the B operand and the in-tile terms there.)
#pragma unroll
          for (int q = 0; q < WT / 4; ++q)
            *yc_quad(p, tau, v, q) = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
      }
    } else if (tid == 128) {
      // ---- planes of every pass through the ring
      for (int k = 0; k < npass && !dead; ++k) {
        const int row0 = wbeg + k * WTM;
        for (int q = 0; q < P && !dead; ++q) {
          const int g = gc + k * P + q, s = g % NS;
          if (g >= NS) bwait(&empty[s], (unsigned)(g / NS - 1) & 1u);
          if (dead) break;
          mbar_arrive_expect_tx(smem_u32(&full[s]), WPLANE);
          tc::tma_load_2d(smem_u32(ahi + s * WPLANE), mapX, q * WPW, row0, smem_u32(&full[s]));
          ++issued[s];
        }
      }
    } else if (tid == 160) {
      // ---- MMAs of every pass into tensor-memory half (pass parity)
      constexpr unsigned id = tc::idesc(WTM, WT, 2);
      for (int k = 0; k < npass && !dead; ++k) {
        const int gpk = gp + k, half = gpk & 1;
        if (gpk >= 2) bwait(&tfree[half], (unsigned)((gpk - 2) >> 1) & 1u);
        tc::fence_after();
        for (int q = 0; q < P && !dead; ++q) {
          const int g = gc + k * P + q, s = g % NS;
          bwait(&loready[s], (unsigned)(g / NS) & 1u);
          if (dead) break;
          tc::fence_after();
          const unsigned a_h = smem_u32(ahi + s * WPLANE), a_l = smem_u32(alo + s * WPLANE);
          const unsigned b_h = smem_u32(bhi + q * WBPLANE), b_l = smem_u32(blo + q * WBPLANE);
          const unsigned d = tmem + (unsigned)((half * P + q) * WT);
#pragma unroll
          for (int kk = 0; kk < WPW / 8; ++kk) {
            const unsigned ko = (unsigned)kk * 32u;
            tc::mma_tf32(d, tc::desc_sw128(a_h + ko), tc::desc_sw128(b_h + ko), id, kk > 0 ? 1u : 0u);
            tc::mma_tf32(d, tc::desc_sw128(a_l + ko), tc::desc_sw128(b_h + ko), id, 1u);
            tc::mma_tf32(d, tc::desc_sw128(a_h + ko), tc::desc_sw128(b_l + ko), id, 1u);
          }
          tc::commit(smem_u32(&empty[s]));
        }
        tc::commit(smem_u32(&done[half]));
      }
    }
    gp += npass;
    gc += npass * P;
    // A claimed block is always published (even after a timed-out wait).
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) red_release_add_gpu(sync_base_done(p, nt, tau), 1);
  }
  // Copies and MMAs still in flight complete before the CTA leaves (bounded).
  if (tid == 128)
    for (int s = 0; s < NS; ++s)
      if (issued[s] > 0) tc::wait(smem_u32(&full[s]), (unsigned)(issued[s] - 1) & 1u, p.wait_ns);
  if (tid == 160) {
    tc::commit(smem_u32(&fin));
    tc::wait(smem_u32(&fin), 0u, p.wait_ns);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, cols);
}

// --------------------------------------------------------------------------
// Chain role: the column chain over all tiles.
// --------------------------------------------------------------------------
template <int RPT>
__device__ void chain_role(const WParams& p, char* smem) {
  constexpr int NW = WNT / 32;
  // The staging buffer, then one mbarrier per column (K of them, each
  // completing once: no re-arming, so a partial that arrives late still
  // lands on its own column's barrier).
  float* st = reinterpret_cast<float*>(smem);                 // RPT x WT x (WNR + 1)
  unsigned long long* cbar = reinterpret_cast<unsigned long long*>(smem + sizeof(float) * RPT * WT * (WNR + 1));
  __shared__ float Gs[2][WT][WT];                             // Q[tile][tile], zero beyond the tile
  __shared__ __align__(16) float Gn[2][WT][WT];               // Q[tile][next tile] of tile tq in Gn[tq & 1]
  __shared__ float wpart[NW];
  __shared__ float cpart[2][WMAXCL];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned rank = cluster_ctarank();
  const int CL = p.cl;
  const int nt = (p.K + WT - 1) / WT;

  // Column g's barrier expects the CL partials of column g (4 bytes each).
  for (int g = tid; g < p.K; g += WNT) {
    mbar_init(smem_u32(&cbar[g]), 1);
    mbar_arrive_expect_tx(smem_u32(&cbar[g]), CL * 4);
  }
  fence_mbar_init();
  __syncthreads();
  cluster_sync_all();                                          // every barrier initialised before any send
  if (tid == 0) red_release_add_gpu(sync_started(p), 1);

  // The two roles of a chain CTA run separate code (their block barriers
  // match one for one): warp 0 exchanges the column partials and publishes
  // the tiles, warps 1 .. NW-1 own the rows.  Keeping them apart leaves the
  // row warps' column loop the whole register file.
  if (warp == 0) {
    for (int tau = 0; tau < nt; ++tau) {
      const int lo = tau * WT, hi = min(p.K, lo + WT), Tw = hi - lo;
      const unsigned cbar_tile = smem_u32(cbar + lo);
      // Blocks of this tile's base that no worker has finished within
      // kGiveUpNs and none has claimed (workers absent or behind): claim
      // them (block w = rank + CL * lane) and compute them here, one row per
      // lane.  The row warps wait for base_done meanwhile.
      if (!(tau == 0 && p.pre0)) {
        const int* bd = sync_base_done(p, nt, tau);
        int need = 0;
        if (lane == 0) {
          const unsigned long long t0 = global_ns();
          unsigned sleep_ns = 32;
          need = ld_acquire_gpu(bd) < p.nb;
          while (need && global_ns() - t0 < kGiveUpNs) {
            __nanosleep(sleep_ns);
            if (sleep_ns < 256) sleep_ns <<= 1;
            need = ld_acquire_gpu(bd) < p.nb;
          }
        }
        need = __shfl_sync(0xffffffffu, need, 0);
        if (need) {
          const int w = (int)rank + CL * lane;
          const bool got = w < p.nb && atomicCAS(sync_state(p, nt, tau, w), 0, 1) == 0;
          const unsigned m = __ballot_sync(0xffffffffu, got);
          if (m) {
            // These blocks read the new columns of tiles <= tau - 2, which
            // every chain CTA has published by now; the acquire makes them
            // visible to this warp.
            if (lane == 0 && tau >= 2) wait_count(sync_chain_done(p, nt, tau - 2), CL, p);
            __syncwarp();
            const int ns = __popc(m);
            for (int e = lane; e < ns * p.per; e += 32) {
              const int i = e / p.per;
              unsigned mm = m;
              for (int k = 0; k < i; ++k) mm &= mm - 1;
              const int v = ((int)rank + CL * (__ffs(mm) - 1)) * p.per + e % p.per;
              if (v < p.N) base_row_global(p, v, lo, hi, tau >= 1 ? lo - WT : 0);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) red_release_add_gpu(sync_base_done(p, nt, tau), ns);
          }
        }
      }
      // Per column: the row warps' partials (block barrier), their sum sent
      // to every CTA of the cluster.  Sent unconditionally (also after a
      // timed-out wait elsewhere), so every column's barrier in every CTA
      // completes and no partial is in flight at exit.  This warp does not
      // need the norm, so it does not wait for the partials.
#pragma unroll
      for (int t = 0; t < WT; ++t) {
        if (t >= Tw) break;
        const int b = t & 1;                                   // partial slot (lo is even)
        __syncthreads();
        // The row warps' partials sit in lanes 1 .. NW - 1 < 16: a butterfly
        // over the low four lane bits gives lanes 0 .. 15 their sum.
        float v = (lane >= 1 && lane < NW) ? wpart[lane] : 0.f;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane < CL) {
          const unsigned raddr = mapa_u32(smem_u32(&cpart[b][rank]), lane);
          const unsigned rbar = mapa_u32(cbar_tile + 8u * t, lane);
          st_async_f32(raddr, v, rbar);
        }
      }
      // Every CTA publishes its own rows (the workers wait for all CL): the
      // block barrier after the row warps' stores, then one release count
      // (cumulative), with no cluster barrier, so no CTA waits for the
      // slowest one here.  The workers read tile tau only for the bases of
      // tiles >= tau + 2.
      __syncthreads();
      if (lane == 0 && (tau + 2 < nt || p.spart)) red_release_add_gpu(sync_chain_done(p, nt, tau), 1);
    }
  } else {
    const int tr = tid - 32;
    // This CTA's rows: the contiguous block [row0, row0 + nloc); local row
    // li = i * WNR + tr belongs to row thread tr, register row i.
    const int row0 = (int)rank * p.chain_rows;
    const int nloc = max(0, min(p.chain_rows, p.N - row0));
    auto sidx = [](int i, int t, int r) { return (i * WT + t) * (WNR + 1) + r; };
    bool valid[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) valid[i] = i * WNR + tr < nloc;
    // y[i][0..15]: the tile's columns (loaded from the tile's base, less
    // the previous tile's contribution).
    float y[RPT][WT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int s = 0; s < WT; ++s) y[i][s] = 0.f;

    // Barrier of the row warps only.  The compiler's named-barrier intrinsic
    // (not inline asm), after an explicit warp reconvergence: a hardware
    // barrier counts a whole warp as arrived when any of its lanes executes
    // it, so a warp split by a divergent wait (thread 32 polls the base
    // flag) would otherwise complete a barrier without its waiting lane.
    auto row_bar = []() {
      __syncwarp();
      __barrier_sync_count(1, WNR);
    };
    // The Q blocks a tile needs are copied asynchronously (cp.async,
    // zero-filled outside the blocks) one tile ahead, off the tile
    // transitions: Gs of tile tq into Gs[tq & 1]; Gn of tile tq (used at the
    // start of tile tq + 1) into Gn[tq & 1].
    auto fetch_gs = [&](int tq) {
      const int qlo = tq * WT, qw = min(p.K, qlo + WT) - qlo;
      for (int e = tr; e < WT * WT; e += WNR) {
        const int i = e / WT, j = e % WT;
        const bool in = i < qw && j < qw;
        cp_async4(&Gs[tq & 1][i][j], p.Q + (in ? (int64_t)(qlo + i) * p.Kp + qlo + j : 0), in);
      }
    };
    auto fetch_gn = [&](int tq) {
      const int qlo = tq * WT, qw = min(p.K, qlo + WT) - qlo;
      const int nlo = qlo + qw, nw = min(p.K, nlo + WT) - nlo;
      for (int e = tr; e < WT * WT; e += WNR) {
        const int i = e / WT, j = e % WT;
        const bool in = i < qw && j < nw;
        cp_async4(&Gn[tq & 1][i][j], p.Q + (in ? (int64_t)(qlo + i) * p.Kp + nlo + j : 0), in);
      }
    };
    fetch_gs(0);
    cp_async_commit();

    bool dead = false;       // a column exchange timed out: skip later exchange waits
    bool base_dead = false;  // a base wait timed out (thread 32): skip later base waits
    for (int tau = 0; tau < nt; ++tau) {
      const int lo = tau * WT, hi = min(p.K, lo + WT), Tw = hi - lo;
      const float(*G)[WT] = Gs[tau & 1];
      const unsigned cbar_tile = smem_u32(cbar + lo);             // column lo + t: cbar_tile + 8 t
      cp_async_wait_all();                                         // Gs of this tile, Gn of the previous one
      // Every block of this tile's base is claimed by a worker that is running
      // and needs nothing more to finish it, or by warp 0 of a chain CTA.  (A
      // timed-out wait is recorded in the status word; later tiles do not
      // wait again.)
      if (tid == 32 && !(tau == 0 && p.pre0) && !base_dead) {
        if (wait_count(sync_base_done(p, nt, tau), p.nb, p) != 1) base_dead = true;
      }
      row_bar();
      // Gn of this tile and Gs of the next: the buffers are free (tile tau - 1
      // finished reading them before the barrier above).
      fetch_gn(tau);
      if (tau + 1 < nt) fetch_gs(tau + 1);
      cp_async_commit();
      if (!(tau == 0 && p.pre0)) {
        // The tile's base for this thread's rows, in its register order: one
        // 16-byte load per register row and column quad (a warp's 512
        // consecutive bytes), all in flight at once.
        const float4* yb = reinterpret_cast<const float4*>(p.Yc) +
                           (((int64_t)(tau & 1) * p.cl + rank) * RPT * 4) * WNR + tr;
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
          for (int q = 0; q < WT / 4; ++q) {
            const float4 v = valid[i] ? yb[(i * 4 + q) * WNR] : make_float4(0.f, 0.f, 0.f, 0.f);
            y[i][4 * q] = v.x;
            y[i][4 * q + 1] = v.y;
            y[i][4 * q + 2] = v.z;
            y[i][4 * q + 3] = v.w;
          }
      } else {
        // Tile 0's base: P, staged through st for this CTA's rows (4 lanes per
        // row, 16 bytes each, 8 loads in flight per thread), plus the early
        // base and its compensation in this thread's register order.
        constexpr int SU = 8;
        const int total = nloc * 4;
        for (int base = tr; base < total; base += SU * WNR) {
          float4 v[SU];
#pragma unroll
          for (int u = 0; u < SU; ++u) {
            const int e = base + u * WNR;
            const int row = row0 + (e >> 2), q = e & 3;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e >= total) continue;
            const int64_t off = (int64_t)row * p.Kp + lo + 4 * q;
            if (4 * q + 3 < Tw) {
              v[u] = *reinterpret_cast<const float4*>(p.P + off);
            } else {
              float w[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) w[j] = 4 * q + j < Tw ? p.P[off + j] : 0.f;
              v[u] = make_float4(w[0], w[1], w[2], w[3]);
            }
          }
#pragma unroll
          for (int u = 0; u < SU; ++u) {
            const int e = base + u * WNR;
            if (e >= total) continue;
            const int li = e >> 2, q = e & 3;
            const int i = li / WNR, r = li - i * WNR;
            st[sidx(i, 4 * q, r)] = v[u].x;
            st[sidx(i, 4 * q + 1, r)] = v[u].y;
            st[sidx(i, 4 * q + 2, r)] = v[u].z;
            st[sidx(i, 4 * q + 3, r)] = v[u].w;
          }
        }
        row_bar();
        // P and the early base cancel: P + early base first (nearly exact),
        // then the early base's compensation.
        const float4* yb = reinterpret_cast<const float4*>(p.Yc) + ((int64_t)rank * RPT * 4) * WNR + tr;
        const float4* cb = reinterpret_cast<const float4*>(p.pre0) + ((int64_t)rank * RPT * 4) * WNR + tr;
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
          for (int q = 0; q < WT / 4; ++q) {
            float4 e = make_float4(0.f, 0.f, 0.f, 0.f), c = e;
            if (valid[i]) {
              e = yb[(i * 4 + q) * WNR];
              c = cb[(i * 4 + q) * WNR];
            }
            const float ev[4] = {e.x, e.y, e.z, e.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
              y[i][4 * q + j] = valid[i] ? (st[sidx(i, 4 * q + j, tr)] + ev[j]) + cv[j] : 0.f;
          }
      }
      if (tau > 0) {
        // The previous tile's contribution, y -= x_prev * Q[prev][tile], for
        // this thread's rows (the previous tile's finished columns still wait
        // in st).  (Unrolled by two: at 4 rows per thread the 4-way unroll
        // spilled 46 / 96 bytes, this 16 / 16, and the text-like K = 160 W
        // update went 298 -> 285 us.)
        // Two columns per instruction (packed FP32 multiply-add, each half
        // rounded as a scalar fmaf).
        const float(*Gp)[WT] = Gn[(tau - 1) & 1];
#pragma unroll 2
        for (int j = 0; j < WT; ++j) {
          float2 nx[RPT];
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const float x = -st[sidx(i, j, tr)];
            nx[i] = make_float2(x, x);
          }
#pragma unroll
          for (int cq = 0; cq < WT / 4; ++cq) {
            const float4 g = *reinterpret_cast<const float4*>(&Gp[j][4 * cq]);
            const float2 g01 = make_float2(g.x, g.y), g23 = make_float2(g.z, g.w);
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
              float2 a = make_float2(y[i][4 * cq], y[i][4 * cq + 1]);
              float2 b = make_float2(y[i][4 * cq + 2], y[i][4 * cq + 3]);
              a = __ffma2_rn(g01, nx[i], a);
              b = __ffma2_rn(g23, nx[i], b);
              y[i][4 * cq] = a.x;
              y[i][4 * cq + 1] = a.y;
              y[i][4 * cq + 2] = b.x;
              y[i][4 * cq + 3] = b.y;
            }
          }
        }
      }

      // Columns t = 0 .. Tw-1 of the tile, unrolled so that every register
      // slot is static: column t is finished and the previous column's
      // contribution is pushed into columns t+1.. (column t already has it);
      // the finished columns wait in st until the tile's end.
      float xp[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) xp[i] = 0.f;
#pragma unroll
      for (int t = 0; t < WT; ++t) {
        if (t >= Tw) break;
        const int b = t & 1;                                     // partial slot (lo is even)
        // The clamped column goes to this thread's slots of st (normalised
        // there after the exchange), keeping registers free across the wait.
        float ss = 0.f;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const float x = fmaxf(p.eps, y[i][t]);
          st[sidx(i, t, tr)] = x;
          if (valid[i]) ss = fmaf(x, x, ss);
        }
        ss = warp_sum(ss);
        if (lane == 0) wpart[warp] = ss;
        __syncthreads();
        if (t > 0) {
          // Columns t+1 .. 15: an odd first one alone, then even-aligned
          // pairs in packed FP32 multiply-adds (each half as a scalar fmaf).
          const int s0 = t + 1;
          if (s0 < WT && (s0 & 1)) {
            const float g = G[t - 1][s0];
#pragma unroll
            for (int i = 0; i < RPT; ++i) y[i][s0] = fmaf(-xp[i], g, y[i][s0]);
          }
#pragma unroll
          for (int s2 = (s0 + 1) & ~1; s2 < WT; s2 += 2) {
            const float2 g = make_float2(G[t - 1][s2], G[t - 1][s2 + 1]);
#pragma unroll
            for (int i = 0; i < RPT; ++i) fma_pair(y[i][s2], y[i][s2 + 1], make_float2(-xp[i], -xp[i]), g);
          }
        }
        // Every row warp waits for the column's CL partials itself and adds
        // them in the same fixed order (no second block barrier): the
        // partials of column lo + t + 2 cannot arrive before every warp here
        // has passed the next column's block barrier, which it does only
        // after reading these.
        if (!dead) {
          const unsigned bar = cbar_tile + 8u * t;
          unsigned long long t0 = 0;
          unsigned polls = 0;
          while (!mbar_try_wait(bar, 0)) {
            if ((++polls & 31u) == 0) {
              const unsigned long long now = global_ns();
              if (t0 == 0) {
                t0 = now;
              } else if (now - t0 > p.wait_ns) {
                dead = true;
                if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
                break;
              }
            }
          }
        }
        dead = __any_sync(0xffffffffu, dead);
        // The CL partials summed by an xor butterfly over lanes 0..15 (lanes
        // 16..31 mirror them): each step adds the same two operands in every
        // lane it pairs, so every lane of every CTA gets the same squared
        // norm.
        float tot = (lane & 15) < CL ? cpart[b][lane & 15] : 0.f;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        const float inv = rsqrtf(tot);                           // 1 / ||column||
        if (tid == 32 && rank == 0 && (!(tot > 0.f) || !(tot < INFINITY))) atomicOr(p.status, ST_NUMERIC);
        const float g1 = t + 1 < WT ? G[t][t + 1] : 0.f;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const float x = st[sidx(i, t, tr)] * inv;
          st[sidx(i, t, tr)] = x;
          if (t + 1 < WT) y[i][t + 1] = fmaf(-x, g1, y[i][t + 1]);
          xp[i] = x;
        }
      }
      // The tile's columns stored once, at its end, then the tile is
      // published (warp 0, after the block barrier; its contribution to the
      // next tile is subtracted at the next tile's start): four lanes per row, so
      // one warp instruction writes eight whole 64-byte row segments
      // (storing four columns of each thread's rows every fourth column
      // wrote a 16-byte piece of 32 rows per instruction and made those
      // columns 2.5x slower: text-like K = 160 W update 283 -> 258 us).
      row_bar();
      if (Tw == WT) {
        // Item e: row li = e / 4 (register row i, thread r), columns 4 (e % 4) ..
#pragma unroll 4
        for (int e = tr; e < nloc * 4; e += WNR) {
          const int li = e >> 2, cq = e & 3;
          const int i = li / WNR, r = li - i * WNR;
          *reinterpret_cast<float4*>(p.X + (int64_t)(row0 + li) * p.Kp + lo + 4 * cq) =
              make_float4(st[sidx(i, 4 * cq, r)], st[sidx(i, 4 * cq + 1, r)], st[sidx(i, 4 * cq + 2, r)],
                          st[sidx(i, 4 * cq + 3, r)]);
        }
      } else {
        for (int e = tr; e < nloc * Tw; e += WNR) {
          const int li = e / Tw, c = e - li * Tw;
          const int i = li / WNR, r = li - i * WNR;
          p.X[(int64_t)(row0 + li) * p.Kp + lo + c] = st[sidx(i, c, r)];
        }
      }
      __syncthreads();
    }
    cp_async_wait_all();                                         // the last tile's Gn (unused)
  }
  // Every CTA has sent every column's partial once it reaches the cluster
  // barrier; each then waits (bounded) until all partials addressed to it
  // have landed, so no remote store is in flight when the cluster leaves.
  __syncthreads();
  cluster_sync_all();
  for (int g = tid; g < p.K; g += WNT) {
    if (!wait_bar_cluster(smem_u32(&cbar[g]), 0, p.wait_ns)) atomicOr(p.status, ST_TIMEOUT);
  }
  // Finished: every row warp's stores precede the block barrier and the
  // release (the worker grid waits for all CL before it ends).
  __syncthreads();
  if (tid == 0) red_release_add_gpu(sync_finished(p, nt), 1);
}

template <int RPT>
__global__ void __launch_bounds__(WNT, 1) w_chain_kernel(WParams p) {
  extern __shared__ __align__(16) char smem[];
  // The worker grid (the next launch, a programmatic dependent) may be
  // scheduled once every CTA of this grid has run this.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  chain_role<RPT>(p, smem);
}

template <int WR, bool TCW>
__global__ void __launch_bounds__(WNT, 1) w_workers_kernel(WParams p, const __grid_constant__ CUtensorMap mapX) {
  extern __shared__ __align__(16) char smem[];
  if (TCW) worker_role_tc(p, smem, (int)blockIdx.x, &mapX);
  else worker_role<WR>(p, smem, (int)blockIdx.x);
  // The grid ends after the chain (bounded wait), so work ordered after it
  // sees the finished factor whatever the two grids' scheduling was.
  __syncthreads();
  if (threadIdx.x == 0) wait_count(sync_finished(p, (p.K + WT - 1) / WT), p.cl, p);
}

size_t chain_smem(int rpt, int Kp) {
  return sizeof(unsigned long long) * (size_t)Kp + sizeof(float) * (size_t)rpt * WT * (WNR + 1);
}
// At least 120 KB, so that two worker CTAs never share an SM (nor a worker
// an SM of the chain): the rows are dealt one block per CTA.
constexpr size_t kWorkerSmemFloor = 120 * 1024;
size_t worker_smem(int Kp, int worker_rows) {
  return std::max(kWorkerSmemFloor,
                  sizeof(float) * ((size_t)(Kp + WT - 1) / WT * WT * WT + (size_t)worker_rows * (Kp + 4)));
}

template <int RPT>
cudaError_t launch_chain_t(const WParams& p, size_t smem, cudaStream_t s) {
  auto kern = w_chain_kernel<RPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.cl, 1, 1);
  cfg.blockDim = dim3(WNT, 1, 1);
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

template <int WR, bool TCW>
cudaError_t launch_workers_t(const WParams& p, const CUtensorMap& map, int n_workers, size_t smem, cudaStream_t s,
                             bool after_chain) {
  auto kern = w_workers_kernel<WR, TCW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_workers, 1, 1);
  cfg.blockDim = dim3(WNT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  // A programmatic dependent of the chain grid: it may begin while the
  // chain runs (it does not wait for the chain grid's completion).  With
  // after_chain, plain stream order instead.
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = after_chain ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kern, p, map);
}

template <int RPT>
int max_clusters_t(int cl, size_t smem) {
  auto kern = w_chain_kernel<RPT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(WNT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int max_clusters(int rpt, int cl, size_t smem) {
  switch (rpt) {
    case 1: return max_clusters_t<1>(cl, smem);
    case 2: return max_clusters_t<2>(cl, smem);
    case 3: return max_clusters_t<3>(cl, smem);
    case 4: return max_clusters_t<4>(cl, smem);
    default: return 0;
  }
}

}  // namespace

size_t w_sync_ints(int K) {
  const size_t nt = (size_t)(K + WT - 1) / WT;
  return (1 + 2 * nt) * kSyncStride + nt * WMAXNB + 2 * kSyncStride;
}

size_t w_sync_sdone_offset(int K) {
  const size_t nt = (size_t)(K + WT - 1) / WT;
  return (1 + 2 * nt) * kSyncStride + nt * WMAXNB;
}

void w_persistent_blocks(int N, const WPersistConfig& cfg, int* nb, int* per) {
  *per = (N + cfg.n_workers - 1) / cfg.n_workers;
  *nb = (N + *per - 1) / *per;
}

bool w_persistent_config(int N, int Kp, WPersistConfig* cfg, bool tc) {
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (int cl : {16, 8}) {
    const int nrc = (N + cl - 1) / cl;
    const int rpt = (nrc + WNR - 1) / WNR;
    if (rpt > 4) continue;
    const int n_workers = std::min(WMAXNB, n_sm - cl);
    if (n_workers < 1) continue;
    // Rows per worker pass: as many (up to 4 lanes per thread's row, a
    // multiple of 8) as the shared-memory budget holds, so that at large K
    // most of the CTA's threads still have a row (K = 400: 120 rows, where
    // halving from 128 gave 64 and left half the threads idle).
    constexpr size_t kBudget = 216 * 1024;
    int worker_rows = WNT / 4;
    while (worker_rows > 16 && worker_smem(Kp, worker_rows) > kBudget) worker_rows -= 8;
    size_t wsmem = worker_smem(Kp, worker_rows);
    if (tc) wsmem = std::max(wsmem, wtc_smem(Kp));      // tensor-core workers: plane ring and B operand
    const size_t csmem = chain_smem(rpt, Kp);
    if (wsmem > kBudget || csmem > kBudget) continue;
    if (max_clusters(rpt, cl, csmem) < 1) continue;
    cfg->cluster = cl;
    cfg->rpt = rpt;
    cfg->chain_rows = nrc;
    cfg->n_workers = n_workers;
    cfg->worker_rows = worker_rows;
    // A worker stages its whole row block at once where it fits (the base
    // is then formed in passes of worker_rows over it, and the block stays
    // in shared memory for the Gram partial).
    {
      const int per = (N + n_workers - 1) / n_workers;
      const size_t whole = sizeof(float) * ((size_t)(Kp + WT - 1) / WT * WT * WT + (size_t)per * (Kp + 4));
      cfg->stage_rows = worker_rows;
      if (!tc && per > worker_rows && whole <= kBudget) {
        cfg->stage_rows = per;
        wsmem = std::max(wsmem, whole);
      }
    }
    cfg->worker_wr = Kp >= 128 ? 2 : 1;
    cfg->chain_smem = csmem;
    cfg->worker_smem = wsmem;
    cfg->tc = tc;
    return true;
  }
  return false;
}

size_t w_chain_base_floats() { return (size_t)3 * WMAXCL * 4 * WNR * WT; }

ChainOrder w_chain_order(float* Yc, int N, const WPersistConfig& cfg) {
  ChainOrder co;
  co.chain_rows = (N + cfg.cluster - 1) / cfg.cluster;
  co.rpt = cfg.rpt;
  co.base = Yc;
  co.comp = Yc + (size_t)2 * cfg.cluster * cfg.rpt * WNR * WT;
  return co;
}

cudaError_t w_persistent_run(float* X, const float* P, const float* Q, float* Yc, int N, int K, int Kp,
                             float eps, int* d_sync, int* d_status, const WPersistConfig& cfg, cudaStream_t s,
                             const float* pre0, unsigned long long wait_ns, int extra_arrivals, float* spart,
                             cudaEvent_t after_chain) {
  if (N <= 0 || K <= 0) return cudaSuccess;
  if (!Yc || cfg.rpt < 1 || cfg.rpt > 4 || cfg.cluster > WMAXCL || (size_t)cfg.cluster * cfg.rpt * WNR < (size_t)N)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(d_sync, 0, sizeof(int) * w_sync_ints(K), s);
  if (e != cudaSuccess) return e;
  if (cfg.n_workers < 1 || cfg.n_workers > WMAXNB) return cudaErrorInvalidValue;
  int nb = 0, per = 0;
  w_persistent_blocks(N, cfg, &nb, &per);
  if (spart && (cfg.tc || Kp > 256 || (size_t)cfg.worker_rows * (Kp + 4) < 16 * 256)) return cudaErrorInvalidValue;
  WParams p{X, P, Q, N, K, Kp, eps, d_status, d_sync, cfg.cluster, cfg.worker_rows, (N + cfg.cluster - 1) / cfg.cluster,
            nb, per, pre0, wait_ns ? wait_ns : kWaitLimitNs, extra_arrivals, spart,
            std::max(cfg.worker_rows, std::min(cfg.stage_rows, per)), Yc, cfg.rpt};
  CUtensorMap map = {};
  if (cfg.tc && !tma_map_f32(&map, X, N, Kp, Kp, WPW, WTM)) return cudaErrorNotSupported;
  switch (cfg.rpt) {
    case 1: e = launch_chain_t<1>(p, cfg.chain_smem, s); break;
    case 2: e = launch_chain_t<2>(p, cfg.chain_smem, s); break;
    case 3: e = launch_chain_t<3>(p, cfg.chain_smem, s); break;
    case 4: e = launch_chain_t<4>(p, cfg.chain_smem, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (after_chain && (e = cudaEventRecord(after_chain, s)) != cudaSuccess) return e;
  const bool ac = cfg.workers_after_chain;
  if (cfg.tc) return launch_workers_t<1, true>(p, map, cfg.n_workers, cfg.worker_smem, s, ac);
  return cfg.worker_wr == 2 ? launch_workers_t<2, false>(p, map, cfg.n_workers, cfg.worker_smem, s, ac)
                            : launch_workers_t<1, false>(p, map, cfg.n_workers, cfg.worker_smem, s, ac);
}

}  // namespace plnmf
