// Fused H update (Alg. 1's H loop in the tiled order of Alg. 2).
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
#include "devutil.cuh"
#include "internal.cuh"

namespace plnmf {
namespace {

// Rows [row0, row0 + nrows) of X (row stride Kp) into shared memory with row
// stride ldx, one bulk copy (TMA, cp.async.bulk) per row, completed on `bar`.
// Every thread returns once the data has landed (bounded wait; on expiry the
// status word gets ST_TIMEOUT).  Row starts and lengths are multiples of 16
// bytes because Kp and ldx are multiples of 4.
__device__ void stage_rows_bulk(float* dst, int ldx, const float* X, int row0, int nrows, int Kp,
                                unsigned long long* bar, int* status) {
  const unsigned b = smem_u32(bar);
  const unsigned bytes = (unsigned)Kp * 4u;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes * nrows) : "memory");
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst + r * ldx)),
        "l"(X + (int64_t)(row0 + r) * Kp), "r"(bytes), "r"(b)
        : "memory");
  }
  unsigned long long t0 = 0;
  unsigned polls = 0;
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b)
        : "memory");
    if (ok) break;
    if ((++polls & 63u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kWaitLimitNs) {
        atomicOr(status, ST_TIMEOUT);
        break;
      }
    }
  }
}

constexpr int HT = 16;            // tile width

// Gc[j * HT + c] = G[j][lo + c] for j < Kr, c < HT (zero beyond K).  The
// loads are issued in batches of 8 before any store, so a thread does not
// stall on each load in turn (in-order issue).
template <int NT>
__device__ __forceinline__ void stage_gcols(float* Gc, const float* __restrict__ G, int Kp, int K, int lo, int Kr) {
  const int total = Kr * HT;
  for (int base = threadIdx.x; base < total; base += 8 * NT) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT;
      const int j = e / HT, c = e % HT;
      v[u] = (e < total && j < K && lo + c < K) ? __ldg(G + (int64_t)j * Kp + lo + c) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT;
      if (e < total) Gc[e] = v[u];
    }
  }
}
// Asynchronous form of stage_gcols for the H update: 16-byte cp.async copies
// (L2 only) into Gc, committed as one group, so the next tile's block of G
// loads while the current tile computes.  A chunk of 4 columns entirely in
// range is copied; one entirely out of range is zero-filled by the copy
// (source size 0); a chunk straddling K (K not a multiple of 4) is written
// with plain stores, masked.
template <int NT, int LDG = HT>
__device__ __forceinline__ void prefetch_gcols(float* Gc, const float* __restrict__ G, int Kp, int K, int lo, int Kr) {
  const int total = Kr * (HT / 4);
  for (int e = threadIdx.x; e < total; e += NT) {
    const int j = e >> 2, q = e & 3;
    const int c = lo + 4 * q;
    float* d = Gc + j * LDG + 4 * q;
    if (j < K && c < K && c + 3 >= K) {
#pragma unroll
      for (int u = 0; u < 4; ++u) d[u] = c + u < K ? G[(int64_t)j * Kp + c + u] : 0.f;
      continue;
    }
    const bool ok = j < K && c + 3 < K;
    const float* src = ok ? G + (int64_t)j * Kp + c : G;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(d)), "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

constexpr int HL = 4;             // lanes per row
constexpr int HROWS = 64;         // rows per CTA
constexpr int HTHREADS = HROWS * HL;
constexpr int W_PREP_R = 2;       // rows per lane group in w_prep_kernel

// R rows per lane group: each group of 4 lanes owns R rows (4 tile columns per
// lane), so a 16-byte load of S's column block serves R rows.  The grid
// leaves few CTAs per SM (D / 32 R of them), so registers are not what limits
// occupancy: planning for two CTAs per SM lets the compiler keep more loads
// in flight (120 registers at R = 1 instead of 60; text-like K = 160:
// 69.8 -> 66.1 us).
// NG lane groups per CTA (32, or 16 for an even spread of few-row CTAs).
template <int R, int NG>
__global__ void __launch_bounds__(4 * NG, 2) h_update_kernel(float* __restrict__ X, const float* __restrict__ B,
                                                          const float* __restrict__ G, int N, int K, int Kp,
                                                          float eps, int* status, const int* skip,
                                                          const float* dref, double* dpart) {
  if (skip && *skip) return;                              // a converged sweep loop (nmf_warm_h)
  // Shared memory: two Gc buffers (Kr x HT each) = G[j][lo + c] for the
  // current and the next tile, zero beyond K; Xs (32 R x (Kp + 4)) = the CTA's
  // rows, updated in place (row stride Kp + 4 keeps the 8 rows a warp reads at
  // once on distinct banks).
  constexpr int NT = 4 * NG, ROWS = NG * R;
  extern __shared__ __align__(16) float smem[];
  const int Kr = (Kp + HT - 1) / HT * HT;
  const int ldx = Kp + 4;
  float* Xs = smem + 2 * Kr * HT;
  const int tid = threadIdx.x;
  const int sub = tid & (HL - 1);
  const int grp = tid >> 2;                               // 0..NG-1
  const int row0 = blockIdx.x * ROWS;
  const int nrows = min(ROWS, N - row0);
  const unsigned full = 0xffffffffu;
  __shared__ __align__(8) unsigned long long bar;
  prefetch_gcols<NT>(smem, G, Kp, K, 0, Kr);
  stage_rows_bulk(Xs, ldx, X, row0, nrows, Kp, &bar, status);
  // Row i of the group: local row grp + 32 i (so a warp's 8 groups touch 8
  // consecutive rows for each i).
  bool valid[R];
  float* xr[R];
  const float* br[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int rl = grp + NG * i;
    valid[i] = rl < nrows;
    xr[i] = Xs + rl * ldx;
    br[i] = B + (int64_t)(valid[i] ? row0 + rl : row0) * Kp;
  }
  // R values of the current tile, loaded one tile ahead.
  float rb[R][4];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * sub + q;
      rb[i][q] = (valid[i] && c < K) ? __ldg(br[i] + c) : 0.f;
    }

  for (int lo = 0, tb = 0; lo < K; lo += HT, tb ^= 1) {
    const int hi = min(K, lo + HT);
    const float* Gc = smem + tb * Kr * HT;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();                                      // Gc of this tile landed; the other buffer is free
    if (lo + HT < K) prefetch_gcols<NT>(smem + (tb ^ 1) * Kr * HT, G, Kp, K, lo + HT, Kr);
    float acc[R][4];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float4 own = lo + 4 * sub < Kp ? *reinterpret_cast<const float4*>(xr[i] + lo + 4 * sub)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
      const float xown[4] = {own.x, own.y, own.z, own.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cl = 4 * sub + q, c = lo + cl;
        acc[i][q] = 0.f;
        if (valid[i] && c < hi) acc[i][q] = fmaf(1.f - Gc[c * HT + cl], xown[q], rb[i][q]);
      }
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lo + HT + 4 * sub + q;
        rb[i][q] = (valid[i] && c < K) ? __ldg(br[i] + c) : 0.f;
      }
    // Columns outside the tile: j < lo (new) and j >= lo + HT (old), in
    // blocks of HT terms folded into acc with compensation (comp_fold).
    float cmp[R][4], blk[R][4];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) cmp[i][q] = blk[i][q] = 0.f;
    // Four columns j .. j+3 into the block partials.
    auto step = [&](int j) {
      float xs[R][4];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const float4 x4 = *reinterpret_cast<const float4*>(xr[i] + j);
        xs[i][0] = x4.x; xs[i][1] = x4.y; xs[i][2] = x4.z; xs[i][3] = x4.w;
      }
      // Two columns per instruction (packed FP32 multiply-add, each half
      // rounded as a scalar fmaf).
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 g = *reinterpret_cast<const float4*>(Gc + (j + u) * HT + 4 * sub);
        const float2 g01 = make_float2(g.x, g.y), g23 = make_float2(g.z, g.w);
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const float2 xx = make_float2(xs[i][u], xs[i][u]);
          float2 a = make_float2(blk[i][0], blk[i][1]);
          float2 b = make_float2(blk[i][2], blk[i][3]);
          a = __ffma2_rn(g01, xx, a);
          b = __ffma2_rn(g23, xx, b);
          blk[i][0] = a.x;
          blk[i][1] = a.y;
          blk[i][2] = b.x;
          blk[i][3] = b.y;
        }
      }
    };
    auto fold = [&]() {
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) comp_fold(acc[i][q], cmp[i][q], blk[i][q]);
    };
    // Full blocks of HT columns unrolled (constant offsets, loads scheduled
    // ahead); a ragged last block (Kp not a multiple of HT) step by step.
    auto outside = [&](int j0, int j1) {
      int jb = j0;
#pragma unroll 1
      for (; jb + HT <= j1; jb += HT) {
#pragma unroll
        for (int jj = 0; jj < HT; jj += 4) step(jb + jj);
        fold();
      }
      if (jb < j1) {
#pragma unroll 1
        for (int j = jb; j < j1; j += 4) step(j);
        fold();
      }
    };
    outside(0, lo);
    outside(lo + HT < Kp ? lo + HT : Kp, Kp);
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] += cmp[i][q];
    // Old in-tile columns j > c.
#pragma unroll
    for (int i = 0; i < R; ++i) {
      float xo[HT];
#pragma unroll
      for (int q = 0; q < HT / 4; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lo + 4 * q < Kp) v = *reinterpret_cast<const float4*>(xr[i] + lo + 4 * q);
        xo[4 * q] = v.x; xo[4 * q + 1] = v.y; xo[4 * q + 2] = v.z; xo[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int j = 1; j < HT; ++j) {
        // The lane's four values of S's row j in one 16-byte load (four
        // scalar loads cost as many wavefronts and four times the issue).
        const float4 g4 = *reinterpret_cast<const float4*>(Gc + (lo + j) * HT + 4 * sub);
        const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cl = 4 * sub + q;
          if (j > cl) acc[i][q] = fmaf(-gv[q], xo[j], acc[i][q]);
        }
      }
    }
    // Finish the tile's columns in order; each new value is broadcast to the
    // group's lanes and pushed into the later columns.
    float xn[R][4];
#pragma unroll
    for (int t = 0; t < HT; ++t) {
      const int owner = t >> 2, q = t & 3;
      const float4 g4t = *reinterpret_cast<const float4*>(Gc + (lo + t) * HT + 4 * sub);
      const float gt[4] = {g4t.x, g4t.y, g4t.z, g4t.w};
#pragma unroll
      for (int i = 0; i < R; ++i) {
        float v = 0.f;
        if (sub == owner) {
          v = fmaxf(eps, acc[i][q]);
          xn[i][q] = v;
        }
        v = __shfl_sync(full, v, (threadIdx.x & 31 & ~(HL - 1)) + owner);
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          const int c2 = 4 * sub + q2;
          if (c2 > t) acc[i][q2] = fmaf(-gt[q2], v, acc[i][q2]);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if (lo + 4 * sub + 3 < hi) {
        *reinterpret_cast<float4*>(xr[i] + lo + 4 * sub) = make_float4(xn[i][0], xn[i][1], xn[i][2], xn[i][3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = lo + 4 * sub + q;
          if (c < hi) xr[i][c] = xn[i][q];
        }
      }
    }
  }
  __syncthreads();
  {
    const int kq = Kp / 4;
    float4* dst = reinterpret_cast<float4*>(X + (int64_t)row0 * Kp);
    const float4* rf = dref ? reinterpret_cast<const float4*>(dref + (int64_t)row0 * Kp) : nullptr;
    // With dpart: this CTA's sums of (new - ref)^2 and ref^2, ref = dref or
    // the old value (read before it is overwritten): per thread in FP32 (a
    // difference of nearby values is exact), then FP64 in a fixed order.
    float da = 0.f, db = 0.f;
    for (int e = tid; e < nrows * kq; e += NT) {
      const int r = e / kq, q = e % kq;
      const float4 v = *reinterpret_cast<const float4*>(Xs + r * ldx + 4 * q);
      if (dpart) {
        const float4 o = rf ? rf[e] : dst[e];
        const float d0 = v.x - o.x, d1 = v.y - o.y, d2 = v.z - o.z, d3 = v.w - o.w;
        da = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, da))));
        db = fmaf(o.x, o.x, fmaf(o.y, o.y, fmaf(o.z, o.z, fmaf(o.w, o.w, db))));
      }
      dst[e] = v;
    }
    if (dpart) {
      __shared__ double pa[NT / 32], pb[NT / 32];
      double xa = da, xb = db;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        xa += __shfl_xor_sync(full, xa, o);
        xb += __shfl_xor_sync(full, xb, o);
      }
      if ((tid & 31) == 0) {
        pa[tid >> 5] = xa;
        pb[tid >> 5] = xb;
      }
      __syncthreads();
      if (tid == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
          ta += pa[w];
          tb += pb[w];
        }
        dpart[2 * blockIdx.x] = ta;
        dpart[2 * blockIdx.x + 1] = tb;
      }
    }
  }
}

// Row-per-warp form of the H update.  Rows (documents) are independent, so a
// warp owns one row: lane l keeps h_j and R_j for j = l, l + 32, ... (M
// registers each) and the row never leaves registers.  For the tile [lo, hi)
// and its column c = lo + t (owned by the lane that holds j = c):
//   1. every lane adds S[j][c] h_j for all 16 t over its own j outside the
//      tile (new values left of it, old values right of it);
//   2. a reduce-scatter over the warp (xor 16, 8, 4, 2 halving the columns
//      each time, then xor 1) leaves column t's sum in lanes 2t and 2t + 1,
//      and one more shuffle moves it to the column's owner;
//   3. the owner forms y_c = (1 - S_cc) h_c + R_c - sum, then subtracts
//      S[j][c] h_j(old) for the tile's j > c (each old value broadcast in
//      turn), which is Alg. 1's y before the tile's own new values;
//   4. the tile's columns are finished in order: h_c(new) = max(eps, y_c) is
//      broadcast and S[c][c'] h_c(new) subtracted from the later columns c'.
// The same terms as h_update_kernel, in another summation order.  The CTA's
// warps share each tile's 16 columns of S in shared memory (double buffered
// with cp.async, as in h_update_kernel).
template <int M>
__global__ void __launch_bounds__(256) h_update_warp_kernel(float* __restrict__ X, const float* __restrict__ B,
                                                            const float* __restrict__ G, int N, int K, int Kp,
                                                            float eps, const int* skip) {
  if (skip && *skip) return;                              // a converged sweep loop (nmf_warm_h)
  constexpr int NT = 256, WARPS = NT / 32;
  // S block rows padded to 20 floats: the 32 lanes read 32 consecutive rows
  // with 16-byte loads, and an 80-byte stride puts every 8 of them on
  // distinct banks.
  constexpr int LDG = HT + 4;
  extern __shared__ __align__(16) float smem[];
  const int Kr = (Kp + HT - 1) / HT * HT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = blockIdx.x * WARPS + warp;
  const bool valid = row < N;
  const unsigned full = 0xffffffffu;
  prefetch_gcols<NT, LDG>(smem, G, Kp, K, 0, Kr);
  float hj[M], rj[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int j = lane + 32 * m;
    const bool in = valid && j < Kp;
    hj[m] = in ? X[(int64_t)row * Kp + j] : 0.f;
    rj[m] = in ? B[(int64_t)row * Kp + j] : 0.f;
  }
  for (int lo = 0, tb = 0; lo < K; lo += HT, tb ^= 1) {
    const int hi = min(K, lo + HT), Tw = hi - lo;
    const float* Gc = smem + tb * Kr * LDG;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();                                      // this tile's block of S landed; the other buffer is free
    if (lo + HT < K) prefetch_gcols<NT, LDG>(smem + (tb ^ 1) * Kr * LDG, G, Kp, K, lo + HT, Kr);
    // Lane o = (lo % 32) + t owns column t (j = lo + t, register slot mt).
    const int mt = lo >> 5;
    const int t_own = lane - (lo & 31);
    const bool own = t_own >= 0 && t_own < Tw;
    float hold = 0.f, r = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m)
      if (m == mt) {
        hold = hj[m];
        r = rj[m];
        if (own) hj[m] = 0.f;                              // the tile's own j stay out of step 1
      }
    // 1. partial column sums over this lane's j outside the tile
    float p[HT];
#pragma unroll
    for (int t = 0; t < HT; ++t) p[t] = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int j = lane + 32 * m;
      if (j < Kp) {
        const float4* g4 = reinterpret_cast<const float4*>(Gc + j * LDG);
#pragma unroll
        for (int q = 0; q < HT / 4; ++q) {
          const float4 g = g4[q];
          const float2 hh = make_float2(hj[m], hj[m]);
          fma_pair(p[4 * q], p[4 * q + 1], make_float2(g.x, g.y), hh);
          fma_pair(p[4 * q + 2], p[4 * q + 3], make_float2(g.z, g.w), hh);
        }
      }
    }
    // 2. reduce-scatter: after the halving steps lane l holds column l >> 1
#pragma unroll
    for (int k = 0; k < 8; ++k) {                          // xor 16: keep columns [8 b4, 8 b4 + 8)
      const bool up = lane & 16;
      const float send = up ? p[k] : p[k + 8];
      const float recv = __shfl_xor_sync(full, send, 16);
      p[k] = (up ? p[k + 8] : p[k]) + recv;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {                          // xor 8
      const bool up = lane & 8;
      const float send = up ? p[k] : p[k + 4];
      const float recv = __shfl_xor_sync(full, send, 8);
      p[k] = (up ? p[k + 4] : p[k]) + recv;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {                          // xor 4
      const bool up = lane & 4;
      const float send = up ? p[k] : p[k + 2];
      const float recv = __shfl_xor_sync(full, send, 4);
      p[k] = (up ? p[k + 2] : p[k]) + recv;
    }
    {                                                      // xor 2
      const bool up = lane & 2;
      const float send = up ? p[0] : p[1];
      const float recv = __shfl_xor_sync(full, send, 2);
      p[0] = (up ? p[1] : p[0]) + recv;
    }
    p[0] += __shfl_xor_sync(full, p[0], 1);                // the two lanes of a column: same sum
    const float T = __shfl_sync(full, p[0], own ? 2 * t_own : 0);
    // 3. y before the tile's own new values
    const float scc = own ? Gc[(lo + t_own) * LDG + t_own] : 0.f;
    float y = fmaf(1.f - scc, hold, r) - T;
#pragma unroll
    for (int t = 0; t < HT; ++t) {
      if (t >= Tw) break;
      const float ho = __shfl_sync(full, hold, (lo & 31) + t);
      if (own && t_own < t) y = fmaf(-Gc[(lo + t) * LDG + t_own], ho, y);
    }
    // 4. the tile's columns in order
    float hnew = hold;
#pragma unroll
    for (int t = 0; t < HT; ++t) {
      if (t >= Tw) break;
      float v = 0.f;
      if (t_own == t) {
        hnew = fmaxf(eps, y);
        v = hnew;
      }
      v = __shfl_sync(full, v, (lo & 31) + t);
      if (own && t_own > t) y = fmaf(-Gc[(lo + t) * LDG + t_own], v, y);
    }
#pragma unroll
    for (int m = 0; m < M; ++m)
      if (m == mt) hj[m] = own ? hnew : hold;
  }
  if (valid) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int j = lane + 32 * m;
      if (j < Kp) X[(int64_t)row * Kp + j] = hj[m];
    }
  }
}

// Base of one W tile [lo, hi) for the column chain (left-looking form of
// Eqs. 4-6): for every row v and tile column c,
//   Y[v, c] = P[v, c] - sum_{j < new_end} Q[j][c] W[v, j](new)
//                     - sum_{j >= hi} Q[j][c] W[v, j](old)
//                     - sum_{c < j < hi} Q[j][c] W[v, j](old).
// (The W_old * Q_cc initialisation of Alg. 2 cancels the j = c term exactly
// and is left out.)  With new_end = lo this is the complete base; with
// new_end = lo - 16 the previous tile is left out, so the kernel can run
// while the chain is still finishing that tile (columns in [new_end, lo) are
// neither read for the result nor written here), and the chain adds the
// previous tile's contribution itself.  B == nullptr leaves the data term out
// (Y = -sums; the caller adds P later); with Ylo given, the compensation of
// the sum goes to Ylo (N x HT) instead of being rounded into Y, since P and
// the sum cancel when the caller adds them.
template <int R>
__global__ void __launch_bounds__(HTHREADS / R) w_prep_kernel(const float* __restrict__ X, const float* __restrict__ B,
                                                              const float* __restrict__ G, float* __restrict__ Y,
                                                              float* __restrict__ Ylo, int N, int K, int Kp, int lo,
                                                              int new_end, int T, int* status, ChainOrder co) {
  // Shared memory: Gc (Kr x HT) = G[j][lo + c], zero beyond K; Xs = the CTA's
  // rows of X (row stride Kp + 4, see h_update_kernel).  A lane group of
  // four lanes takes R of the CTA's HROWS rows (rows g, g + HROWS / R, ...),
  // so one 16-byte load of Gc serves R rows.
  constexpr int NT = HTHREADS / R;
  constexpr int NGR = NT / HL;                            // lane groups
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) unsigned long long bar;
  const int Kr = (Kp + HT - 1) / HT * HT;
  const int ldx = Kp + 4;
  float* Gc = smem;
  float* Xs = smem + Kr * HT;
  const int hi = min(K, lo + T);                          // tile [lo, hi), T <= HT columns
  const int tid = threadIdx.x;
  const int sub = tid & (HL - 1);
  const int row0 = blockIdx.x * HROWS;
  const int nrows = min(HROWS, N - row0);
  stage_gcols<NT>(Gc, G, Kp, K, lo, Kr);
  stage_rows_bulk(Xs, ldx, X, row0, nrows, Kp, &bar, status);
  if ((tid >> 2) >= nrows) return;                        // (its later rows are out too)
  int lrow[R];
  bool valid[R];
  const float* xr[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    lrow[i] = (tid >> 2) + i * NGR;
    valid[i] = lrow[i] < nrows;
    xr[i] = Xs + lrow[i] * ldx;                           // within the HROWS staged rows
  }
  float acc[R][4];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lo + 4 * sub + q;
      acc[i][q] = (valid[i] && c < hi && B) ? __ldg(B + (int64_t)(row0 + lrow[i]) * Kp + c) : 0.f;
    }
  // Blocks of HT terms folded into acc with compensation (comp_fold).
  float cmp[R][4], blk[R][4];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) cmp[i][q] = blk[i][q] = 0.f;
  auto step = [&](int j) {
    float xs[R][4];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float4 x4 = *reinterpret_cast<const float4*>(xr[i] + j);
      xs[i][0] = x4.x; xs[i][1] = x4.y; xs[i][2] = x4.z; xs[i][3] = x4.w;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 g = *reinterpret_cast<const float4*>(Gc + (j + u) * HT + 4 * sub);
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const float2 xx = make_float2(xs[i][u], xs[i][u]);
        fma_pair(blk[i][0], blk[i][1], make_float2(g.x, g.y), xx);
        fma_pair(blk[i][2], blk[i][3], make_float2(g.z, g.w), xx);
      }
    }
  };
  auto fold = [&]() {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) comp_fold(acc[i][q], cmp[i][q], blk[i][q]);
  };
  // Full blocks unrolled; a ragged last block step by step.
  auto outside = [&](int j0, int j1) {
    int jb = j0;
#pragma unroll 1
    for (; jb + HT <= j1; jb += HT) {
#pragma unroll
      for (int jj = 0; jj < HT; jj += 4) step(jb + jj);
      fold();
    }
    if (jb < j1) {
#pragma unroll 1
      for (int j = jb; j < j1; j += 4) step(j);
      fold();
    }
  };
  outside(0, new_end);
  outside(lo + T < Kp ? lo + T : Kp, Kp);
  // Old in-tile columns j > c: one more block.
#pragma unroll
  for (int i = 0; i < R; ++i) {
    float xo[HT];
#pragma unroll
    for (int q = 0; q < HT / 4; ++q) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (lo + 4 * q < Kp) v = *reinterpret_cast<const float4*>(xr[i] + lo + 4 * q);
      xo[4 * q] = v.x; xo[4 * q + 1] = v.y; xo[4 * q + 2] = v.z; xo[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 1; j < HT; ++j) {
      const float4 g4 = *reinterpret_cast<const float4*>(Gc + (lo + j) * HT + 4 * sub);
      const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cl = 4 * sub + q;
        if (j > cl && j < T) blk[i][q] = fmaf(gv[q], xo[j], blk[i][q]);
      }
    }
  }
  fold();
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (!valid[i]) continue;
    const int row = row0 + lrow[i];
    if (co.base) {
      // In the W chain's register order (lo = 0, T = 16: this lane's quad;
      // zero past K, where every G factor is).
      const long long qi = chain_quad(row, sub, co.chain_rows, co.rpt);
      reinterpret_cast<float4*>(co.base)[qi] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      reinterpret_cast<float4*>(co.comp)[qi] = make_float4(cmp[i][0], cmp[i][1], cmp[i][2], cmp[i][3]);
      continue;
    }
    float* yr = Y + (int64_t)row * Kp;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lo + 4 * sub + q;
      if (c >= hi) continue;
      if (Ylo) {
        yr[c] = acc[i][q];
        Ylo[(int64_t)row * HT + c - lo] = cmp[i][q];
      } else {
        yr[c] = acc[i][q] + cmp[i][q];
      }
    }
  }
}

}  // namespace

cudaError_t w_prep_run(const float* X, const float* B, const float* G, float* Y, int N, int K, int Kp, int lo,
                       int new_end, int* status, cudaStream_t s, int T, float* Ylo, const ChainOrder* co) {
  if (T < 1 || T > HT) return cudaErrorInvalidValue;
  if (co && (B || lo != 0 || new_end != 0 || T != HT || !co->base || !co->comp || co->chain_rows < 1 || co->rpt < 1))
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * ((size_t)((Kp + HT - 1) / HT * HT) * HT + (size_t)HROWS * (Kp + 4));
  const int blocks = (N + HROWS - 1) / HROWS;
  auto kern = w_prep_kernel<W_PREP_R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, HTHREADS / W_PREP_R, smem, s>>>(X, B, G, Y, B ? nullptr : Ylo, N, K, Kp, lo, new_end, T, status,
                                                  co ? *co : ChainOrder{});
  return cudaGetLastError();
}

template <int R, int NG = 32>
cudaError_t h_update_launch(float* X, const float* B, const float* G, int N, int K, int Kp, float eps, int* status,
                            cudaStream_t s, const int* skip, const float* dref = nullptr, double* dpart = nullptr,
                            int* nblk = nullptr) {
  const size_t smem = sizeof(float) * (2 * (size_t)((Kp + HT - 1) / HT * HT) * HT + (size_t)NG * R * (Kp + 4));
  auto kern = h_update_kernel<R, NG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (N + NG * R - 1) / (NG * R);
  if (nblk) *nblk = blocks;
  kern<<<blocks, 4 * NG, smem, s>>>(X, B, G, N, K, Kp, eps, status, skip, dref, dpart);
  return cudaGetLastError();
}

template <int M>
cudaError_t h_update_warp_launch(float* X, const float* B, const float* G, int N, int K, int Kp, float eps,
                                 cudaStream_t s, const int* skip) {
  const size_t smem = sizeof(float) * 2 * (size_t)((Kp + HT - 1) / HT * HT) * (HT + 4);
  auto kern = h_update_warp_kernel<M>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(N + 7) / 8, 256, smem, s>>>(X, B, G, N, K, Kp, eps, skip);
  return cudaGetLastError();
}

namespace {
cudaError_t h_update_dispatch(float* X, const float* B, const float* G, int N, int K, int Kp, float eps,
                              int* status, cudaStream_t s, const int* skip, const float* dref, double* dpart,
                              int* nblk, bool pack_rows = false) {
  // One warp per row for short rows (Kp <= 32): the row is one register per
  // lane and the warp kernel's per-row column chain is short.  For longer
  // rows the four-lanes-per-row kernel is faster: its chain runs for eight
  // rows per warp at once (measured at K = 160: 68 us against 96 us).
  if ((Kp + 31) / 32 == 1) {
    if (dpart) return cudaErrorInvalidValue;              // (h_update_sweep checks this form separately)
    return h_update_warp_launch<1>(X, B, G, N, K, Kp, eps, s, skip);
  }
  // Four lanes per row, rows per lane group chosen for occupancy.
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  const size_t per_row = sizeof(float) * (size_t)(Kp + 4);
  const size_t gc = sizeof(float) * (size_t)((Kp + HT - 1) / HT * HT) * HT;
  auto fits = [&](int R) { return 2 * gc + per_row * 32 * R <= 200 * 1024; };
  auto enough = [&](int R) { return (long long)(N + 32 * R - 1) / (32 * R) >= 3LL * sms; };
  if (fits(4) && enough(4)) return h_update_launch<4>(X, B, G, N, K, Kp, eps, status, s, skip, dref, dpart, nblk);
  if (fits(2) && enough(2)) return h_update_launch<2>(X, B, G, N, K, Kp, eps, status, s, skip, dref, dpart, nblk);
  // Long rows: two or three rows per lane group even with few CTAs, as one
  // 16-byte load of S's block then serves them all (8192 x 256: 115 -> 101 us;
  // at K = 160 one row is faster, 66 against 68 us on 11,314 rows).  Of the
  // two, the one with the fewer waves x rows per CTA: where a 64-row CTA
  // needs more than half the shared memory the 2-row grid runs in two waves
  // and the 3-row grid in one.
  if (Kp >= 192 && fits(2)) {
    auto cost = [&](int R) -> long long {
      const size_t bytes = 2 * gc + per_row * 32 * R;
      const long long per_sm = std::max<long long>(1, (long long)(227 * 1024) / (long long)bytes);
      const long long blocks = (N + 32 * R - 1) / (32 * R);
      return (blocks + per_sm * sms - 1) / (per_sm * sms) * R;
    };
    if (2 * gc + per_row * 96 <= 220 * 1024 && cost(3) < cost(2))
      return h_update_launch<3>(X, B, G, N, K, Kp, eps, status, s, skip, dref, dpart, nblk);
    return h_update_launch<2>(X, B, G, N, K, Kp, eps, status, s, skip, dref, dpart, nblk);
  }
  // 16-group CTAs spread more evenly over the SMs than 32-group ones (11,314
  // rows, one row per group: 708 CTAs, 4.8 per SM, against 354 at 2.4 per
  // SM: 66.6 -> 64.1 us at K = 160).  Two rows per group where that still
  // leaves a CTA per SM: a 16-byte load of S's block then serves both rows,
  // and the kernel is bound by its shared-memory wavefronts (11,314 rows at
  // K = 160: 60.3 -> 56.2 us; 8,000 rows at K = 128: 37.5 -> 33.3 us).
  if (pack_rows || (long long)(N + 31) / 32 >= sms)
    return h_update_launch<2, 16>(X, B, G, N, K, Kp, eps, status, s, skip, dref, dpart, nblk);
  return h_update_launch<1, 16>(X, B, G, N, K, Kp, eps, status, s, skip, dref, dpart, nblk);
}
}  // namespace

cudaError_t h_update_run(float* X, const float* B, const float* G, int N, int K, int Kp, float eps,
                         int* status, cudaStream_t s, const int* skip, bool pack_rows) {
  if (N <= 0 || K <= 0) return cudaSuccess;
  return h_update_dispatch(X, B, G, N, K, Kp, eps, status, s, skip, nullptr, nullptr, nullptr, pack_rows);
}

size_t h_sweep_partials(int N) { return 2 * (size_t)((N + 15) / 16); }

cudaError_t h_update_sweep(float* X, const float* B, const float* G, int N, int K, int Kp, float eps, int* status,
                           cudaStream_t s, const float* Href, float* Hprev, double* part, float tol, int sweep,
                           double* trace, int* state) {
  if (N <= 0 || K <= 0) return cudaErrorInvalidValue;
  if ((Kp + 31) / 32 == 1) {
    // The row-per-warp form has no epilogue: the previous sweep's H is kept
    // in Hprev and the change is formed by a pass of its own.
    cudaError_t e;
    if (!Href && (e = copy_unless_done(Hprev, X, (int64_t)N * Kp, state, s)) != cudaSuccess) return e;
    if ((e = h_update_warp_launch<1>(X, B, G, N, K, Kp, eps, s, state)) != cudaSuccess) return e;
    return diff_check(X, Href ? Href : Hprev, N, K, Kp, part, tol, sweep, trace, state, s);
  }
  int nblk = 0;
  cudaError_t e = h_update_dispatch(X, B, G, N, K, Kp, eps, status, s, state, Href, part, &nblk);
  if (e != cudaSuccess) return e;
  return sweep_check(part, nblk, tol, sweep, trace, state, s);
}

}  // namespace plnmf
