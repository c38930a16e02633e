// nmf_gram_noalloc: the Gram matrix S = X^T X without any device allocation.
//
// The split-N partial sums that the Gram kernel needs live in one file-scope
// device array of fixed size instead of memory obtained from cudaMalloc.
// Host code cannot use the array's name as a device address (it is a host
// stand-in for the symbol), so the first call on each device asks the
// runtime for the address with cudaGetSymbolAddress while that device is
// current, and every call passes that address to the kernels.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace plnmf {
namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_gram_scratch[NMF_NOALLOC_SCRATCH_FLOATS];

std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Address of the scratch array on the current device (looked up once per
// device).  Returns nullptr if the lookup fails.
float* scratch_for_current_device(cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *err = cudaSuccess;
  return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace plnmf

extern "C" nmf_status nmf_gram_noalloc(const float* X, int32_t N, int32_t K, int64_t ldx, float* S, void* stream) {
  using namespace plnmf;
  if (!X || !S || N <= 0 || K <= 0 || ldx < K) return NMF_EINVAL;
  const long long kk = (long long)K * K;
  if (kk > NMF_NOALLOC_SCRATCH_FLOATS) return NMF_EUNSUPPORTED;       // one partial must fit
  cudaError_t err;
  float* part = scratch_for_current_device(&err);
  if (!part) return NMF_ECUDA;
  // Split the N rows into chunks: about two waves of work, within the array.
  const int tiles = ((K + 63) / 64) * ((K + 63) / 64 + 1) / 2;
  int want = (296 + tiles - 1) / tiles;
  if (want < 1) want = 1;
  const long long max_chunks = NMF_NOALLOC_SCRATCH_FLOATS / kk;
  if (want > max_chunks) want = (int)max_chunks;
  // Rows per chunk: a multiple of 16, at least N / max_chunks so that the
  // chunks' partials fit the array.
  const long long need = ((long long)N + max_chunks - 1) / max_chunks;
  long long chunk = std::max<long long>(((long long)N + want - 1) / want, need);
  chunk = std::max<long long>(16, (chunk + 15) / 16 * 16);
  const int n_chunks = (int)((N + chunk - 1) / chunk);
  err = gram_run_scratch(X, N, K, ldx, part, n_chunks, (int)chunk, S, static_cast<cudaStream_t>(stream));
  return err == cudaSuccess ? NMF_OK : NMF_ECUDA;
}
