// H update (Alg. 1's H loop in the tiled order of Alg. 2) with the off-tile
// sums of every tile (Eqs. 4 and 6: the contributions of the new columns
// left of the tile and of the old columns right of it) on the tensor cores.
//
// For a tile [lo, lo + 16) and a row h of H^T, column c of the tile starts
// from
//   y_c = R_c + (1 - S_cc) h_c - sum_{j outside the tile} S[j][c] h_j
//         - sum_{c < j < lo + 16} S[j][c] h_j(old)
// with h_j already new left of the tile (rows are independent: no
// normalisation), and the tile's 16 columns are then finished in order, each
// clamped at eps and pushed into the later ones (Eq. 5).  The off-tile sum of
// 128 rows is a [128 x Kp] x [Kp x 16] product with the tile's own rows of S
// masked to zero; it runs on tcgen05 in FP32 accuracy: both operands split
// as x = hi + lo with hi = tf32(x) and lo = tf32(x - hi), three kind::tf32
// MMAs per K step (hi hi + lo hi + hi lo, about 2^-21 relative per product),
// each 32-column plane of the row accumulated in its own 16-column slice of
// tensor memory, and the planes' partial sums folded into the running value
// with compensation (TwoSum, as the SIMT kernel folds its 16-term blocks).
//
// One CTA per 128 rows, 256 threads:
//  * warps 0-3 (one thread per row, TMEM lane = row): split each streamed
//    plane of their rows into hi and lo, fold the slices, run the tile's
//    column chain and write the new columns back;
//  * thread 128: streams the 32-column planes of the CTA's rows of H^T
//    (TMA, 128-byte swizzle) through a ring of up to 6 slots;
//  * thread 160: issues the MMAs of each plane once it is split and commits;
//  * warps 6-7: build the masked, split B operand of the next tile into the
//    other of two buffers while the current tile's MMAs run.
// The planes of the next tile are streamed while the current tile's chain
// runs, the one holding the current tile's columns last: only it has to wait
// until they are written back (they are part of the next tile's sums).  Every
// wait is bounded: on expiry the
// status word gets ST_TIMEOUT and the thread stops waiting; before leaving,
// copies and MMAs still in flight are waited for (bounded) and the tensor
// memory is freed.
#include <algorithm>

#include "devutil.cuh"
#include "internal.cuh"
#include "tcutil.cuh"

namespace plnmf {
namespace {

constexpr int TM = 128;             // rows per CTA (TMEM lanes)
constexpr int HT = 16;              // tile width
constexpr int PW = 32;              // FP32 columns per plane (128 bytes)
constexpr int NSMAX = 6;            // ring slots at most
constexpr int PLANE = TM * 128;     // bytes of one plane of A (16 KB)
constexpr int BPLANE = HT * 128;    // bytes of one plane of B (2 KB)
constexpr int NTHR = 256;
constexpr int kProducer = 128;      // warp 4, lane 0
constexpr int kIssuer = 160;        // warp 5, lane 0
constexpr int kBuild0 = 192;        // warps 6-7
constexpr int kNBuild = NTHR - kBuild0;

struct HtcParams {
  float* X;              // N x Kp (H^T), old on entry, new on exit
  const float* B;        // N x Kp (R)
  const float* G;        // Kp x Kp (S, symmetric)
  int N, K, Kp;
  float eps;
  int* status;
  unsigned long long wait_ns;
};

__host__ __device__ constexpr unsigned tmem_cols_for(int P) {
  return P * HT <= 32 ? 32u : P * HT <= 64 ? 64u : P * HT <= 128 ? 128u : P * HT <= 256 ? 256u : 512u;
}

// Plane streamed k-th for tile tau: the plane holding tile tau - 1's columns
// (written back just before) comes last, the others in order.
__host__ __device__ inline int plane_order(int tau, int k, int P) {
  if (tau == 0) return k;
  const int dep = ((tau - 1) * HT) / PW;
  return k < P - 1 ? (k < dep ? k : k + 1) : dep;
}

// Ring slots: as many planes as fit beside the two B buffers (at most one
// tile's worth, at most NSMAX, at least 2).
__host__ __device__ constexpr int htc_slots(int Kp) {
  return (Kp + PW - 1) / PW < 2 ? 2
         : ((200 * 1024 - 4 * ((Kp + PW - 1) / PW) * BPLANE) / (2 * PLANE) < ((Kp + PW - 1) / PW < NSMAX ? (Kp + PW - 1) / PW : NSMAX)
                ? (200 * 1024 - 4 * ((Kp + PW - 1) / PW) * BPLANE) / (2 * PLANE)
                : ((Kp + PW - 1) / PW < NSMAX ? (Kp + PW - 1) / PW : NSMAX));
}

size_t htc_smem(int Kp) {
  const int P = (Kp + PW - 1) / PW;
  return (size_t)2 * htc_slots(Kp) * PLANE + (size_t)4 * P * BPLANE + 1024;
}

__global__ void __launch_bounds__(NTHR, 1) h_update_tc_kernel(const __grid_constant__ CUtensorMap mapX, HtcParams p) {
  extern __shared__ __align__(1024) char smem_raw[];
  char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int P = (p.Kp + PW - 1) / PW;
  const int NS = htc_slots(p.Kp);
  char* ahi = smem;                         // NS planes: hi (split in place)
  char* alo = smem + NS * PLANE;            // NS planes: lo
  // Two B buffers (tile parity), each P planes of hi then P planes of lo.
  char* bbuf = smem + 2 * NS * PLANE;
  __shared__ __align__(8) unsigned long long full[NSMAX], loready[NSMAX], empty[NSMAX];
  // done: tile tau's MMAs complete (row threads); bfree[b]: the MMAs of the
  // last tile that read B buffer b complete (builders; one barrier per buffer
  // so that a parity wait can never be two phases behind).
  __shared__ __align__(8) unsigned long long done, bready[2], bfree[2], written, fin;
  __shared__ unsigned tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row0 = blockIdx.x * TM;
  const int nt = (p.K + HT - 1) / HT;
  const unsigned cols = tmem_cols_for(P);

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&loready[s]), TM);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    mbar_init(smem_u32(&bready[0]), kNBuild);
    mbar_init(smem_u32(&bready[1]), kNBuild);
    mbar_init(smem_u32(&bfree[0]), 1);
    mbar_init(smem_u32(&bfree[1]), 1);
    mbar_init(smem_u32(&written), TM);
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

  if (tid < TM) {
    // ---- row threads ------------------------------------------------------
    const int row = row0 + tid;
    const bool valid = row < p.N;
    float* xrow = p.X + (int64_t)(valid ? row : 0) * p.Kp;
    const float* brow = p.B + (int64_t)(valid ? row : 0) * p.Kp;
    const unsigned lane_base = (unsigned)(warp * 32) << 16;
    for (int tau = 0; tau < nt; ++tau) {
      const int lo = tau * HT, w = min(p.K, lo + HT) - lo;
      // Old values and R of the tile's columns (zero past the tile).
      float xo[HT], acc[HT], cmp[HT];
#pragma unroll
      for (int c = 0; c < HT; ++c) {
        const bool in = valid && c < w;
        xo[c] = in ? xrow[lo + c] : 0.f;
        const float r = in ? __ldg(brow + lo + c) : 0.f;
        const float scc = c < w ? __ldg(p.G + (int64_t)(lo + c) * p.Kp + lo + c) : 0.f;
        acc[c] = in ? fmaf(1.f - scc, xo[c], r) : 0.f;
        cmp[c] = 0.f;
      }
      // Split each plane of this row as it arrives (streaming order): hi =
      // tf32(x) in place, lo = tf32(x - hi).
      for (int k = 0; k < P; ++k) {
        const int g = tau * P + k, s = g % NS;
        bwait(&full[s], (unsigned)(g / NS) & 1u);
        char* ph = ahi + s * PLANE;
        char* pl = alo + s * PLANE;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const unsigned off = tc::sw128_off(tid, u * 16);
          const float4 v = *reinterpret_cast<const float4*>(ph + off);
          float4 h, l;
          h.x = tc::tf32_rn(v.x); l.x = tc::tf32_rn(v.x - h.x);
          h.y = tc::tf32_rn(v.y); l.y = tc::tf32_rn(v.y - h.y);
          h.z = tc::tf32_rn(v.z); l.z = tc::tf32_rn(v.z - h.z);
          h.w = tc::tf32_rn(v.w); l.w = tc::tf32_rn(v.w - h.w);
          *reinterpret_cast<float4*>(ph + off) = h;
          *reinterpret_cast<float4*>(pl + off) = l;
        }
        tc::fence_async_smem();
        mbar_arrive(smem_u32(&loready[s]));
      }
      // The planes' partial sums (slice q = plane q), folded in plane order.
      bwait(&done, (unsigned)tau & 1u);
      tc::fence_after();
      for (int q = 0; q < P; ++q) {
        float blk[HT];
        tc::tmem_ld16(tmem + lane_base + (unsigned)(q * HT), blk);
#pragma unroll
        for (int c = 0; c < HT; ++c) comp_fold(acc[c], cmp[c], blk[c]);
      }
      tc::fence_before();
#pragma unroll
      for (int c = 0; c < HT; ++c) acc[c] += cmp[c];
      // Old in-tile columns j > c, then the column chain.
      const float* gt = p.G + (int64_t)lo * p.Kp + lo;
#pragma unroll
      for (int j = 1; j < HT; ++j) {
#pragma unroll
        for (int c = 0; c < HT; ++c)
          if (j > c && j < w) acc[c] = fmaf(-__ldg(gt + (int64_t)j * p.Kp + c), xo[j], acc[c]);
      }
      float xn[HT];
#pragma unroll
      for (int t = 0; t < HT; ++t) {
        xn[t] = fmaxf(p.eps, acc[t]);
#pragma unroll
        for (int c = 0; c < HT; ++c)
          if (c > t && t < w && c < w) acc[c] = fmaf(-__ldg(gt + (int64_t)t * p.Kp + c), xn[t], acc[c]);
      }
      if (valid) {
        if (w == HT) {
#pragma unroll
          for (int q = 0; q < HT / 4; ++q)
            *reinterpret_cast<float4*>(xrow + lo + 4 * q) =
                make_float4(xn[4 * q], xn[4 * q + 1], xn[4 * q + 2], xn[4 * q + 3]);
        } else {
          for (int c = 0; c < w; ++c) xrow[lo + c] = xn[c];
        }
      }
      // The next tile's planes (loaded by TMA) read these columns.
      fence_proxy_async_global();
      mbar_arrive(smem_u32(&written));
    }
  } else if (tid == kProducer) {
    // ---- TMA producer -----------------------------------------------------
    int issued[NSMAX] = {0, 0, 0, 0, 0, 0};
    for (int tau = 0; tau < nt && !dead; ++tau) {
      for (int k = 0; k < P && !dead; ++k) {
        const int g = tau * P + k, s = g % NS;
        // The last plane of a tile holds the previous tile's columns.
        if (tau >= 1 && k == P - 1) bwait(&written, (unsigned)(tau - 1) & 1u);
        if (g >= NS) bwait(&empty[s], (unsigned)(g / NS - 1) & 1u);
        if (dead) break;
        mbar_arrive_expect_tx(smem_u32(&full[s]), PLANE);
        tc::tma_load_2d(smem_u32(ahi + s * PLANE), &mapX, plane_order(tau, k, P) * PW, row0, smem_u32(&full[s]));
        ++issued[s];
      }
    }
    // Copies still in flight land before the CTA leaves (bounded).
    for (int s = 0; s < NS; ++s)
      if (issued[s] > 0) tc::wait(smem_u32(&full[s]), (unsigned)(issued[s] - 1) & 1u, p.wait_ns);
  } else if (tid == kIssuer) {
    // ---- MMA issuer -------------------------------------------------------
    constexpr unsigned id = tc::idesc(TM, HT, 2);
    for (int tau = 0; tau < nt && !dead; ++tau) {
      bwait(&bready[tau & 1], (unsigned)(tau >> 1) & 1u);
      tc::fence_after();
      const char* bhi = bbuf + (tau & 1) * 2 * P * BPLANE;
      const char* blo = bhi + P * BPLANE;
      for (int k = 0; k < P && !dead; ++k) {
        const int g = tau * P + k, s = g % NS;
        const int q = plane_order(tau, k, P);                // plane q -> TMEM slice q
        bwait(&loready[s], (unsigned)(g / NS) & 1u);
        if (dead) break;
        tc::fence_after();
        const unsigned a_h = smem_u32(ahi + s * PLANE), a_l = smem_u32(alo + s * PLANE);
        const unsigned b_h = smem_u32(bhi + q * BPLANE), b_l = smem_u32(blo + q * BPLANE);
        const unsigned d = tmem + (unsigned)(q * HT);
#pragma unroll
        for (int kk = 0; kk < PW / 8; ++kk) {
          const unsigned ko = (unsigned)kk * 32u;
          tc::mma_tf32(d, tc::desc_sw128(a_h + ko), tc::desc_sw128(b_h + ko), id, kk > 0 ? 1u : 0u);
          tc::mma_tf32(d, tc::desc_sw128(a_l + ko), tc::desc_sw128(b_h + ko), id, 1u);
          tc::mma_tf32(d, tc::desc_sw128(a_h + ko), tc::desc_sw128(b_l + ko), id, 1u);
        }
        tc::commit(smem_u32(&empty[s]));
      }
      tc::commit(smem_u32(&done));
      tc::commit(smem_u32(&bfree[tau & 1]));
    }
    // Every MMA issued has completed before the tensor memory is freed.
    tc::commit(smem_u32(&fin));
    tc::wait(smem_u32(&fin), 0u, p.wait_ns);
  } else if (tid >= kBuild0) {
    // ---- B operand of each tile: B[c][j] = S[lo + c][j] (= S[j][lo + c]),
    // zero inside the tile and past K, split into hi and lo ---------------
    const int bt = tid - kBuild0;
    const int W = P * PW;
    for (int tau = 0; tau < nt; ++tau) {
      const int lo = tau * HT;
      // Buffer tau & 1 was last read by the MMAs of tile tau - 2 (phase
      // (tau - 2) / 2 of its barrier).
      if (tau >= 2) bwait(&bfree[tau & 1], (unsigned)((tau - 2) >> 1) & 1u);
      char* bhi = bbuf + (tau & 1) * 2 * P * BPLANE;
      char* blo = bhi + P * BPLANE;
      for (int e = bt; e < HT * W; e += kNBuild) {
        const int c = e / W, j = e % W;
        const bool in = j < p.K && lo + c < p.K && !(j >= lo && j < lo + HT);
        const float v = in ? __ldg(p.G + (int64_t)(lo + c) * p.Kp + j) : 0.f;
        const float h = tc::tf32_rn(v), l = tc::tf32_rn(v - h);
        const unsigned off = (unsigned)((j / PW) * BPLANE) + tc::sw128_off(c, (j % PW) * 4);
        *reinterpret_cast<float*>(bhi + off) = h;
        *reinterpret_cast<float*>(blo + off) = l;
      }
      tc::fence_async_smem();
      mbar_arrive(smem_u32(&bready[tau & 1]));
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, cols);
}

}  // namespace

bool h_update_tc_supported(int Kp) { return Kp >= HT && Kp <= kMaxK && htc_smem(Kp) <= 227 * 1024; }

cudaError_t h_update_tc_run(float* X, const float* B, const float* G, int N, int K, int Kp, float eps, int* status,
                            cudaStream_t s) {
  if (N <= 0 || K <= 0) return cudaSuccess;
  if (!h_update_tc_supported(Kp)) return cudaErrorInvalidValue;
  CUtensorMap map;
  if (!tma_map_f32(&map, X, N, Kp, Kp, PW, TM)) return cudaErrorNotSupported;
  const size_t smem = htc_smem(Kp);
  static const cudaError_t attr = [] {
    size_t most = 0;                                   // the largest request over every supported Kp
    for (int kp = HT; kp <= kMaxK; kp += 4) most = std::max(most, htc_smem(kp));
    return cudaFuncSetAttribute(h_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
  }();
  if (attr != cudaSuccess) return attr;
  HtcParams prm{X, B, G, N, K, Kp, eps, status, kWaitLimitNs};
  h_update_tc_kernel<<<(N + TM - 1) / TM, NTHR, smem, s>>>(map, prm);
  return cudaGetLastError();
}

}  // namespace plnmf
