// Learned warm start for the fixed-W H subproblem: a small network maps a new
// document's data term r = W^T a (one row of R = A^T W, Alg. 1) to an
// initial h, from which the H loop of Alg. 1 (S = W^T W fixed) is
// repeated.  The paper has no learned component; the network is fixed here:
//   z1 = x W1 + b1, a1 = GELU(z1), z2 = a1 W2 + b2, a2 = GELU(z2),
//   z3 = a2 W3 + b3, y = softplus(z3)       (Wl stored n_in x n_out)
// with GELU in the exact erf form and softplus(x) = x above 20.  Training
// minimises the mean squared error to the converged h* with Adam.
//
// Arithmetic: the three matrix products of the forward pass and the six of
// the backward pass run on the tensor cores (the TMA-fed BF16 kernel, FP32
// accumulation); the master weights, Adam moments, pre-activations and all
// elementwise work stay FP32.  Each product is C = A B^T with both operands
// K-major, so the weights are kept in BF16 in both layouts (Wl^T for the
// forward product, Wl for the input gradient) and activations / gradients
// are transposed to BF16 where the batch is the contraction dimension.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "internal.cuh"

namespace plnmf {
namespace {

constexpr float kSoftplusThreshold = 20.f;

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}
__device__ __forceinline__ float softplus_f(float x) { return x > kSoftplusThreshold ? x : log1pf(expf(x)); }
__device__ __forceinline__ float softplus_grad_f(float x) {
  return x > kSoftplusThreshold ? 1.f : 1.f / (1.f + expf(-x));
}

// z (rows x n, row stride ldz) += bias; a = act(z) into `a` (row stride lda).
// act 0 = GELU, 1 = softplus.
__global__ void bias_act_kernel(float* __restrict__ z, int64_t ldz, const float* __restrict__ bias, int rows, int n,
                                int act, float* __restrict__ a, int64_t lda) {
  const int64_t total = (int64_t)rows * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n;
    const int c = (int)(e - r * n);
    const float v = z[r * ldz + c] + bias[c];
    z[r * ldz + c] = v;
    a[r * lda + c] = act == 0 ? gelu_f(v) : softplus_f(v);
  }
}

// Output layer gradient of the mean squared error over rows x n outputs:
// dz = 2 (y - t) / (rows n) * softplus'(z); per-block partial sums of the
// squared error (FP64) for the loss.
__global__ void out_grad_kernel(const float* __restrict__ z, const float* __restrict__ y,
                                const float* __restrict__ t, int rows, int n, float* __restrict__ dz,
                                double* __restrict__ part) {
  __shared__ double sh[256];
  const int64_t total = (int64_t)rows * n;
  const float scale = 2.f / (float)total;
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[e] - t[e];
    s += (double)d * (double)d;
    dz[e] = scale * d * softplus_grad_f(z[e]);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// dz = da * GELU'(z), all rows x n contiguous.
__global__ void hidden_grad_kernel(const float* __restrict__ da, const float* __restrict__ z, int64_t total,
                                   float* __restrict__ dz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    dz[e] = da[e] * gelu_grad_f(z[e]);
}

// out[c] = sum over rows of M[r][c] (rows in ascending order).
__global__ void colsum_kernel(const float* __restrict__ M, int rows, int n, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += M[(int64_t)r * n + c];
  out[c] = s;
}

// One Adam step on n parameters.  The coefficients 1 - b1, 1 - b2 and the
// bias corrections 1 - b1^t, 1 - b2^t come from the host (computed in
// double), so that at t = 1 the corrected moments are g and g^2 up to one
// rounding each.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float c1, float c2,
                            float eps, float bc1, float bc2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + c1 * gi;
    const float vi = b2 * v[e] + c2 * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// Sum of (H - Href)^2 and of Href^2 (or of H^2 when Href is null) over rows x
// K of two row-stride-ld buffers (ld a multiple of 4): a warp per row at a
// time, 16-byte loads, each lane's squares summed in FP32 (a difference of
// two nearby FP32 values is exact, its square within one rounding; FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU), then
// FP64 across lanes and warps in a fixed order, one pair of partials per
// block.
__global__ void diff_norm_kernel(const float* __restrict__ H, const float* __restrict__ Href, int rows, int K,
                                 int ld, double* __restrict__ part, const int* skip) {
  if (skip && *skip) return;
  __shared__ double sa[8], sb[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K4 = (K + 3) / 4;
  float a = 0.f, b = 0.f;
  for (int r = blockIdx.x * 8 + warp; r < rows; r += gridDim.x * 8) {
    const float4* hr = reinterpret_cast<const float4*>(H + (int64_t)r * ld);
    const float4* qr = Href ? reinterpret_cast<const float4*>(Href + (int64_t)r * ld) : nullptr;
    for (int c4 = lane; c4 < K4; c4 += 32) {
      const float4 h = hr[c4];
      const float4 q = qr ? qr[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float hv[4] = {h.x, h.y, h.z, h.w}, qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (4 * c4 + u >= K) break;
        const float d = hv[u] - qv[u];
        a = fmaf(d, d, a);
        b = qr ? fmaf(qv[u], qv[u], b) : fmaf(hv[u], hv[u], b);
      }
    }
  }
  double da = a, db = b;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    da += __shfl_xor_sync(0xffffffffu, da, o);
    db += __shfl_xor_sync(0xffffffffu, db, o);
  }
  if (lane == 0) {
    sa[warp] = da;
    sb[warp] = db;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < 8; ++w) {
      ta += sa[w];
      tb += sb[w];
    }
    part[2 * blockIdx.x] = ta;
    part[2 * blockIdx.x + 1] = tb;
  }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(1184, std::max<int64_t>(1, (n + 255) / 256)); }

// The partials summed (256 threads, each a strided subset in order, then a
// fixed tree), the relative change recorded, the loop marked done at tol.
__global__ void diff_check_kernel(const double* __restrict__ part, int nblk, float tol, int sweep,
                                  double* __restrict__ trace, int* __restrict__ state) {
  if (state[0]) return;
  __shared__ double sa[256], sb[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 256) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  a = sa[0];
  b = sb[0];
  const double val = b > 0.0 ? sqrt(a / b) : sqrt(a);
  trace[sweep - 1] = val;
  state[1] = sweep;
  if (val <= (double)tol) state[0] = 1;
}

__global__ void copy_unless_done_kernel(float4* __restrict__ dst, const float4* __restrict__ src, int64_t n4,
                                        const int* __restrict__ state) {
  if (state[0]) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

__global__ void scale_shift_kernel(float* __restrict__ x, int64_t n, float a, float b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = fmaf(a, x[e], b);
}

}  // namespace

// x = a x + b elementwise.
cudaError_t scale_shift(float* x, int64_t n, float a, float b, cudaStream_t s) {
  scale_shift_kernel<<<grid_for(n), 256, 0, s>>>(x, n, a, b);
  return cudaGetLastError();
}

constexpr int kDiffBlocks = 296;

cudaError_t diff_norm(const float* H, const float* Href, int rows, int K, int ld, double* d_part, double* h_out,
                      cudaStream_t s) {
  diff_norm_kernel<<<kDiffBlocks, 256, 0, s>>>(H, Href, rows, K, ld, d_part, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double host[2 * kDiffBlocks];
  if ((e = cudaMemcpyAsync(host, d_part, sizeof(host), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < kDiffBlocks; ++i) {
    a += host[2 * i];
    b += host[2 * i + 1];
  }
  h_out[0] = a;
  h_out[1] = b;
  return cudaSuccess;
}

size_t diff_norm_partials() { return 2 * kDiffBlocks; }

cudaError_t diff_check(const float* H, const float* Href, int rows, int K, int ld, double* d_part, float tol,
                       int sweep, double* trace, int* state, cudaStream_t s) {
  diff_norm_kernel<<<kDiffBlocks, 256, 0, s>>>(H, Href, rows, K, ld, d_part, state);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sweep_check(d_part, kDiffBlocks, tol, sweep, trace, state, s);
}

cudaError_t sweep_check(const double* d_part, int nblk, float tol, int sweep, double* trace, int* state,
                        cudaStream_t s) {
  diff_check_kernel<<<1, 256, 0, s>>>(d_part, nblk, tol, sweep, trace, state);
  return cudaGetLastError();
}

cudaError_t copy_unless_done(float* dst, const float* src, int64_t n, const int* state, cudaStream_t s) {
  if (n % 4) return cudaErrorInvalidValue;
  copy_unless_done_kernel<<<grid_for(n / 4), 256, 0, s>>>(reinterpret_cast<float4*>(dst),
                                                          reinterpret_cast<const float4*>(src), n / 4, state);
  return cudaGetLastError();
}

}  // namespace plnmf

using namespace plnmf;

// Network: dims {K, hidden, hidden, K}; parameters [W1, b1, W2, b2, W3, b3],
// Wl row-major n_in x n_out.
struct nmf_mlp {
  int K = 0, hidden = 0;
  int dims[4] = {0, 0, 0, 0};
  int ldin = 0;                       // BF16 row stride of the input (K rounded up to 8)
  float* p[6] = {};                   // FP32 master parameters
  float* m[6] = {};                   // Adam first moments
  float* v[6] = {};                   // Adam second moments
  float* g[6] = {};                   // gradients
  void* wT[3] = {};                   // BF16 Wl^T, n_out x ld(n_in)
  void* w[3] = {};                    // BF16 Wl, n_in x ld(n_out)
  int64_t t = 0;                      // Adam steps taken
  int* d_status = nullptr;
  // activations / gradients for up to `cap` rows
  int cap = 0;
  float* z[3] = {};                   // pre-activations (FP32), rows x n_out
  float* a[3] = {};                   // activations (FP32), rows x n_out (a[2] = y)
  void* ab[3] = {};                   // BF16 layer inputs: x, a1, a2 (rows x ld)
  void* abT[3] = {};                  // BF16 transposed layer inputs (n_in x ld8(rows))
  float* dz = nullptr;                // rows x max n
  float* da = nullptr;                // rows x max n
  void* dzb = nullptr;                // BF16 dz (rows x max n)
  void* dzT = nullptr;                // BF16 dz^T (max n x ld8(rows))
  double* part = nullptr;             // loss partials
  float* xin = nullptr;               // staged input (rows x K) when the caller's is not contiguous
};

namespace {

constexpr int kLossBlocks = 296;

int r8(int x) { return (x + 7) / 8 * 8; }
int64_t nparams(const nmf_mlp* n, int i) {
  const int l = i / 2;
  return (i % 2 == 0) ? (int64_t)n->dims[l] * n->dims[l + 1] : n->dims[l + 1];
}

void free_acts(nmf_mlp* n) {
  for (int l = 0; l < 3; ++l) {
    cudaFree(n->z[l]);
    cudaFree(n->a[l]);
    cudaFree(n->ab[l]);
    cudaFree(n->abT[l]);
    n->z[l] = n->a[l] = nullptr;
    n->ab[l] = n->abT[l] = nullptr;
  }
  cudaFree(n->dz);
  cudaFree(n->da);
  cudaFree(n->dzb);
  cudaFree(n->dzT);
  cudaFree(n->xin);
  n->xin = nullptr;
  n->dz = n->da = nullptr;
  n->dzb = n->dzT = nullptr;
  n->cap = 0;
}

cudaError_t ensure_cap(nmf_mlp* n, int rows) {
  if (rows <= n->cap) return cudaSuccess;
  free_acts(n);
  const int cap = std::max(rows, 1024);
  const int maxn = std::max(n->K, n->hidden);
  cudaError_t e;
  for (int l = 0; l < 3; ++l) {
    const int nin = n->dims[l], nout = n->dims[l + 1];
    const int ldi = l == 0 ? n->ldin : nin;
    if ((e = cudaMalloc(&n->z[l], sizeof(float) * (size_t)cap * nout)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&n->a[l], sizeof(float) * (size_t)cap * nout)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&n->ab[l], 2 * (size_t)cap * ldi)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&n->abT[l], 2 * (size_t)nin * r8(cap))) != cudaSuccess) return e;
  }
  if ((e = cudaMalloc(&n->dz, sizeof(float) * (size_t)cap * maxn)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&n->da, sizeof(float) * (size_t)cap * maxn)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&n->dzb, 2 * (size_t)cap * maxn)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&n->dzT, 2 * (size_t)maxn * r8(cap))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&n->xin, sizeof(float) * (size_t)cap * n->K)) != cudaSuccess) return e;
  n->cap = cap;
  return cudaSuccess;
}

// BF16 copies of the weights in both layouts, from the FP32 masters.
cudaError_t refresh_bf16(nmf_mlp* n, cudaStream_t s) {
  for (int l = 0; l < 3; ++l) {
    const int nin = n->dims[l], nout = n->dims[l + 1];
    const int ldi = l == 0 ? n->ldin : nin;
    cudaError_t e = transpose_to_bf16(n->p[2 * l], nin, nout, nout, n->wT[l], ldi, s);   // nout x ldi
    if (e != cudaSuccess) return e;
    if ((e = convert_bf16(n->p[2 * l], nin, nout, nout, n->w[l], nout, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Forward pass of `rows` inputs (x rows x K, row stride ldx, FP32, device);
// y = a[2] (rows x K).
cudaError_t forward_impl(nmf_mlp* n, const float* x, int64_t ldx, int rows, cudaStream_t s) {
  cudaError_t e = ensure_cap(n, rows);
  if (e != cudaSuccess) return e;
  if ((e = convert_bf16(x, rows, n->K, ldx, n->ab[0], n->ldin, s)) != cudaSuccess) return e;
  for (int l = 0; l < 3; ++l) {
    const int nin = n->dims[l], nout = n->dims[l + 1];
    const int ldi = l == 0 ? n->ldin : nin;
    // z = input * Wl  ==  input (rows x nin) * (Wl^T)^T
    if ((e = tc_bf16_tma_gemm(n->ab[l], ldi, n->wT[l], ldi, n->z[l], nout, rows, nout, nin, n->d_status, s)) !=
        cudaSuccess)
      return e;
    bias_act_kernel<<<grid_for((int64_t)rows * nout), 256, 0, s>>>(n->z[l], nout, n->p[2 * l + 1], rows, nout,
                                                                    l == 2 ? 1 : 0, n->a[l], nout);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l < 2 && (e = convert_bf16(n->a[l], rows, nout, nout, n->ab[l + 1], nout, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Backward pass after forward_impl; targets t (rows x K, contiguous).
// Gradients into g[]; the summed squared error into *sse (synchronous read).
cudaError_t backward_impl(nmf_mlp* n, const float* t, int rows, double* sse, cudaStream_t s) {
  const int K = n->K;
  cudaError_t e;
  out_grad_kernel<<<kLossBlocks, 256, 0, s>>>(n->z[2], n->a[2], t, rows, K, n->dz, n->part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int ldr = r8(rows);
  for (int l = 2; l >= 0; --l) {
    const int nin = n->dims[l], nout = n->dims[l + 1];
    // dz (rows x nout) is current.  gWl = input^T dz = (input^T) (dz^T)^T
    if ((e = transpose_to_bf16(n->dz, rows, nout, nout, n->dzT, ldr, s)) != cudaSuccess) return e;
    const float* in = l == 0 ? nullptr : n->a[l - 1];
    if (l == 0) {
      // the input is held only in BF16; its transpose is built from the FP32 copy
      if ((e = transpose_to_bf16(n->xin, rows, nin, nin, n->abT[0], ldr, s)) != cudaSuccess) return e;
    } else if ((e = transpose_to_bf16(in, rows, nin, nin, n->abT[l], ldr, s)) != cudaSuccess) {
      return e;
    }
    if ((e = tc_bf16_tma_gemm(n->abT[l], ldr, n->dzT, ldr, n->g[2 * l], nout, nin, nout, rows, n->d_status, s)) !=
        cudaSuccess)
      return e;
    colsum_kernel<<<(nout + 127) / 128, 128, 0, s>>>(n->dz, rows, nout, n->g[2 * l + 1]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l == 0) break;
    // da = dz Wl^T = dz (rows x nout) * (Wl)^T with Wl (nin x nout) K-major
    if ((e = convert_bf16(n->dz, rows, nout, nout, n->dzb, nout, s)) != cudaSuccess) return e;
    if ((e = tc_bf16_tma_gemm(n->dzb, nout, n->w[l], nout, n->da, nin, rows, nin, nout, n->d_status, s)) !=
        cudaSuccess)
      return e;
    hidden_grad_kernel<<<grid_for((int64_t)rows * nin), 256, 0, s>>>(n->da, n->z[l - 1], (int64_t)rows * nin,
                                                                      n->dz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (sse) {
    std::vector<double> host(kLossBlocks);
    if ((e = cudaMemcpyAsync(host.data(), n->part, sizeof(double) * kLossBlocks, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double acc = 0.0;
    for (double v : host) acc += v;
    *sse = acc;
  }
  return cudaSuccess;
}

nmf_status st_from(cudaError_t e) {
  if (e == cudaSuccess) return NMF_OK;
  if (e == cudaErrorMemoryAllocation) return NMF_ENOMEM;
  if (e == cudaErrorInvalidValue) return NMF_EINVAL;
  if (e == cudaErrorNotSupported) return NMF_EUNSUPPORTED;
  return NMF_ECUDA;
}

void free_mlp(nmf_mlp* n) {
  if (!n) return;
  cudaDeviceSynchronize();
  free_acts(n);
  for (int i = 0; i < 6; ++i) {
    cudaFree(n->p[i]);
    cudaFree(n->m[i]);
    cudaFree(n->v[i]);
    cudaFree(n->g[i]);
  }
  for (int l = 0; l < 3; ++l) {
    cudaFree(n->wT[l]);
    cudaFree(n->w[l]);
  }
  cudaFree(n->d_status);
  cudaFree(n->part);
  delete n;
}

}  // namespace

// Entry points used by the context code (fixed-W warm start).
namespace plnmf {
cudaError_t mlp_forward_dev(nmf_mlp* n, const float* x, int64_t ldx, int rows, float* y, int64_t ldy,
                            cudaStream_t s) {
  cudaError_t e = forward_impl(n, x, ldx, rows, s);
  if (e != cudaSuccess) return e;
  return cudaMemcpy2DAsync(y, sizeof(float) * ldy, n->a[2], sizeof(float) * n->K, sizeof(float) * n->K, rows,
                           cudaMemcpyDefault, s);
}
int mlp_K(const nmf_mlp* n) { return n->K; }
int mlp_status(const nmf_mlp* n) {
  int st = 0;
  cudaMemcpy(&st, n->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  return st;
}
}  // namespace plnmf

extern "C" {

nmf_status nmf_mlp_create(int32_t K, int32_t hidden, uint64_t seed, nmf_mlp** out) {
  // Row strides of the BF16 operands must be multiples of 8 elements (TMA).
  if (!out || K < 8 || (K & 7) || hidden < 8 || (hidden & 7)) return NMF_EINVAL;
  *out = nullptr;
  if (!tma_available()) return NMF_EUNSUPPORTED;
  nmf_mlp* n = new (std::nothrow) nmf_mlp;
  if (!n) return NMF_ENOMEM;
  n->K = K;
  n->hidden = hidden;
  n->dims[0] = K;
  n->dims[1] = hidden;
  n->dims[2] = hidden;
  n->dims[3] = K;
  n->ldin = r8(K);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
    const size_t b = sizeof(float) * (size_t)nparams(n, i);
    if ((e = cudaMalloc(&n->p[i], b)) != cudaSuccess) break;
    if ((e = cudaMalloc(&n->m[i], b)) != cudaSuccess) break;
    if ((e = cudaMalloc(&n->v[i], b)) != cudaSuccess) break;
    if ((e = cudaMalloc(&n->g[i], b)) != cudaSuccess) break;
    cudaMemset(n->m[i], 0, b);
    cudaMemset(n->v[i], 0, b);
    cudaMemset(n->g[i], 0, b);
  }
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    const int nin = n->dims[l], nout = n->dims[l + 1];
    const int ldi = l == 0 ? n->ldin : nin;
    if ((e = cudaMalloc(&n->wT[l], 2 * (size_t)nout * ldi)) != cudaSuccess) break;
    e = cudaMalloc(&n->w[l], 2 * (size_t)nin * nout);
  }
  if (e == cudaSuccess) e = cudaMalloc(&n->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&n->part, sizeof(double) * kLossBlocks);
  if (e != cudaSuccess) {
    free_mlp(n);
    return st_from(e);
  }
  // He-uniform weights, W ~ U(-sqrt(6 / n_in), sqrt(6 / n_in)), from the
  // SplitMix64 stream of `seed` (layer l uses seed + l); zero biases.
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    const int nin = n->dims[l], nout = n->dims[l + 1];
    if ((e = fill_uniform_splitmix(n->p[2 * l], nin, nout, nout, seed + (uint64_t)l, nullptr)) != cudaSuccess) break;
    if ((e = scale_shift(n->p[2 * l], (int64_t)nin * nout, 2.f * sqrtf(6.f / nin), -sqrtf(6.f / nin), nullptr)) !=
        cudaSuccess)
      break;
    e = cudaMemset(n->p[2 * l + 1], 0, sizeof(float) * nout);
  }
  if (e == cudaSuccess) e = refresh_bf16(n, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_mlp(n);
    return st_from(e);
  }
  *out = n;
  return NMF_OK;
}

nmf_status nmf_mlp_set_params(nmf_mlp* n, const float* const* params) {
  if (!n || !params) return NMF_EINVAL;
  for (int i = 0; i < 6; ++i) {
    if (!params[i]) return NMF_EINVAL;
    const cudaError_t e = cudaMemcpy(n->p[i], params[i], sizeof(float) * nparams(n, i), cudaMemcpyDefault);
    if (e != cudaSuccess) return st_from(e);
  }
  const cudaError_t e = refresh_bf16(n, nullptr);
  if (e != cudaSuccess) return st_from(e);
  return st_from(cudaDeviceSynchronize());
}

nmf_status nmf_mlp_get_params(nmf_mlp* n, float* const* params) {
  if (!n || !params) return NMF_EINVAL;
  for (int i = 0; i < 6; ++i) {
    if (!params[i]) return NMF_EINVAL;
    const cudaError_t e = cudaMemcpy(params[i], n->p[i], sizeof(float) * nparams(n, i), cudaMemcpyDefault);
    if (e != cudaSuccess) return st_from(e);
  }
  return NMF_OK;
}

nmf_status nmf_mlp_forward(nmf_mlp* n, const float* X, int32_t rows, float* Y, void* stream) {
  if (!n || !X || !Y || rows < 0) return NMF_EINVAL;
  if (rows == 0) return NMF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = mlp_forward_dev(n, X, n->K, rows, Y, n->K, s);
  if (e != cudaSuccess) return st_from(e);
  return NMF_OK;
}

nmf_status nmf_mlp_grads(nmf_mlp* n, const float* X, const float* T, int32_t rows, float* const* grads,
                         double* loss) {
  if (!n || !X || !T || rows < 1) return NMF_EINVAL;
  cudaError_t e = ensure_cap(n, rows);
  if (e == cudaSuccess) e = cudaMemcpy(n->xin, X, sizeof(float) * (size_t)rows * n->K, cudaMemcpyDefault);
  if (e == cudaSuccess) e = forward_impl(n, n->xin, n->K, rows, nullptr);
  double sse = 0.0;
  if (e == cudaSuccess) e = backward_impl(n, T, rows, &sse, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return st_from(e);
  if (loss) *loss = sse / ((double)rows * n->K);
  if (grads)
    for (int i = 0; i < 6; ++i)
      if (grads[i] && (e = cudaMemcpy(grads[i], n->g[i], sizeof(float) * nparams(n, i), cudaMemcpyDefault)) !=
                          cudaSuccess)
        return st_from(e);
  return mlp_status(n) ? NMF_ETIMEOUT : NMF_OK;
}

nmf_status nmf_mlp_train_step(nmf_mlp* n, const float* X, const float* T, int32_t rows, float lr, double* loss,
                              void* stream) {
  if (!n || !X || !T || rows < 1 || !(lr > 0.f)) return NMF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_cap(n, rows);
  if (e != cudaSuccess) return st_from(e);
  if ((e = cudaMemcpyAsync(n->xin, X, sizeof(float) * (size_t)rows * n->K, cudaMemcpyDefault, s)) != cudaSuccess)
    return st_from(e);
  if ((e = forward_impl(n, n->xin, n->K, rows, s)) != cudaSuccess) return st_from(e);
  double sse = 0.0;
  if ((e = backward_impl(n, T, rows, loss ? &sse : nullptr, s)) != cudaSuccess) return st_from(e);
  n->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = (float)(1.0 - std::pow(b1, (double)n->t)), bc2 = (float)(1.0 - std::pow(b2, (double)n->t));
  for (int i = 0; i < 6; ++i) {
    const int64_t cnt = nparams(n, i);
    adam_kernel<<<grid_for(cnt), 256, 0, s>>>(n->p[i], n->g[i], n->m[i], n->v[i], cnt, lr, (float)b1, (float)b2,
                                               (float)(1.0 - b1), (float)(1.0 - b2), 1e-8f, bc1, bc2);
    if ((e = cudaGetLastError()) != cudaSuccess) return st_from(e);
  }
  if ((e = refresh_bf16(n, s)) != cudaSuccess) return st_from(e);
  if (loss) *loss = sse / ((double)rows * n->K);
  return NMF_OK;
}

void nmf_mlp_destroy(nmf_mlp* n) { free_mlp(n); }

}  // extern "C"
