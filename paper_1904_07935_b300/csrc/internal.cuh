// Internal declarations shared by the CUDA translation units of libplnmf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/nmf.h"

namespace plnmf {

// Device status word bits (set by kernels, read and cleared by the host).
enum : int {
  ST_TIMEOUT = 1,   // a bounded spin-wait gave up
  ST_NUMERIC = 2,   // a column norm was zero or not finite
};

// Wall-clock limit of every device-side wait (read from %globaltimer).  The
// waits inside one iteration last microseconds; a wait that exceeds this
// sets ST_TIMEOUT in the status word and the kernel stops waiting.
constexpr unsigned long long kWaitLimitNs = 200ull * 1000ull * 1000ull;

constexpr int kMaxK = 512;

// ---------------------------------------------------------------------------
// SpMM (CSR times tall dense) with a host-built, deterministic work plan.
// ---------------------------------------------------------------------------
struct SpmmPlan {
  int rows = 0, cols = 0;
  int n_items = 0;          // work items {row, nnz_begin, nnz_end, slot}
  int n_long = 0;           // rows split into several items
  int n_slots = 0;          // partial rows written by split items
  int4* d_items = nullptr;
  int4* d_combine = nullptr;  // {row, first_slot, n_slots, 0}
  float* d_partial = nullptr; // n_slots x Kp
  int* d_slot_long = nullptr; // long-row index of each slot
  int* d_counter = nullptr;   // per long row: items done in this launch (the last resets it)
};

// Builds the plan from host CSR row pointers.  seg = max nnz per item.
cudaError_t spmm_plan_build(SpmmPlan& plan, const std::vector<int>& row_ptr, int rows, int cols,
                            int Kp, int seg);
void spmm_plan_free(SpmmPlan& plan);
// Y (rows x Kp) = A (CSR) * X (cols x Kp).
cudaError_t spmm_run(const SpmmPlan& plan, const int* col_idx, const float* val, const float* X,
                     float* Y, int Kp, cudaStream_t s);

// ---------------------------------------------------------------------------
// SIMT FP32 GEMM family (64 x 64 CTA tiles, 4 x 4 register micro-tiles).
// ---------------------------------------------------------------------------
enum GemmMode : int {
  GM_STORE = 0,     // C = acc
  GM_PHASE1 = 1,    // C = E + c'_n * X[m][n] - acc  (strictly-upper masked B)
  GM_SUB = 2,       // C -= acc
  GM_PARTIAL = 3,   // C[z] = acc over k-chunk z (split-K partials)
  GM_RESID2 = 4,    // dpart[block] = sum over the tile of (E - acc)^2 (FP64)
};

struct GemmArgs {
  int M = 0, N = 0, Kin = 0;
  const float* A = nullptr;  int64_t lda = 0;  int transA = 0;   // op(A)[m][k]
  const float* B = nullptr;  int64_t ldb = 0;  int transB = 0;   // B[k][n] (or B[n][k] if transB)
  float* C = nullptr;        int64_t ldc = 0;
  int mode = GM_STORE;
  // GM_PHASE1 extras: E (M x N, lde), X (M x N, ldx) and the Gram G whose
  // diagonal gives c'_n = h_mode ? 1 - G[n][n] : 0.  The mask keeps B[k][n]
  // only for k > n (global indices).
  const float* E = nullptr;  int64_t lde = 0;
  const float* X = nullptr;  int64_t ldx = 0;
  int h_mode = 0;
  // GM_PARTIAL: k-range of chunk z is [z*k_chunk, (z+1)*k_chunk); partial z
  // starts at C + z * part_stride.
  int k_chunk = 0;  int64_t part_stride = 0;  int n_chunks = 1;
  // Only tiles with (tile_n >= tile_m) are computed when upper_only (Grams).
  int upper_only = 0;
  double* dpart = nullptr;   // GM_RESID2: one FP64 partial per CTA (grid.x * grid.y)
};

cudaError_t gemm_run(const GemmArgs& a, cudaStream_t s);

// Tensor-core (tcgen05) version of the same family; upper_only is not
// supported.  a_bf16: optional BF16 copy of A with A's layout (BF16 mode).
enum TcPrecision : int { TC_TF32X3 = 0, TC_BF16 = 1 };
cudaError_t tc_gemm_run(const GemmArgs& g, TcPrecision prec, const void* a_bf16, int bn, int* d_status,
                        cudaStream_t s);
int tc_pick_bn(int N);

// BF16 products with TMA-fed tcgen05 MMAs: C (M x N, FP32) = A (M x Kd) B (N x Kd)^T,
// A and B BF16, K-major, row strides lda / ldb multiples of 8 elements.
bool tma_available();
// A_lo != nullptr: A split, C = (A + A_lo) B^T with A_lo of A's layout (A =
// bf16 of the FP32 values, A_lo = bf16 of the remainder); B_lo != nullptr as
// well: C = A B^T + A_lo B^T + A B_lo^T.
cudaError_t tc_bf16_tma_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int M,
                             int N, int Kd, int* d_status, cudaStream_t s, const void* A_lo = nullptr,
                             const void* B_lo = nullptr);
// Split-K partial Grams of X (N x Kp) given X^T in BF16 (Kp x ldx, ldx a
// multiple of 8): part[z] (Kp x Kp) = X^T X over the z-th K slice,
// z < splits (tma_gram_splits gives a full-GPU count); sum with gram_reduce.
// Xt_lo != nullptr: the factor split (X_hi X_hi^T + X_lo X_hi^T + X_hi X_lo^T).
cudaError_t tc_bf16_tma_gram_partials(const void* Xt, int64_t ldx, int Kp, int N, float* part, int splits,
                                      int* d_status, cudaStream_t s, const void* Xt_lo = nullptr);
int tma_gram_splits(int Kp, int N);
// S (Kp x Kp, pads zero) = sum of n_chunks partial Grams, FP64 in a fixed
// order, upper triangle mirrored.
cudaError_t gram_reduce(const float* part, int n_chunks, int Kp, int K, float* S, cudaStream_t s);
// Split-K for products whose tile grid leaves SMs idle: K slices per
// product (1 = no split) and the split run, partials in part
// (n_chunks x M x N floats) summed into a.C in a fixed order.
int splitk_chunks(int M, int N, int Kin);
cudaError_t gemm_run_split(GemmArgs a, float* part, int n_chunks, cudaStream_t s);
// dst (cols x ldd, BF16) = transpose of src (rows x cols FP32, row stride lds); rows..ldd zero.
// lo != nullptr: also lo = bf16(src - dst) in dst's layout (split form).
cudaError_t transpose_to_bf16(const float* src, int rows, int cols, int64_t lds, void* dst, int64_t ldd,
                              cudaStream_t s, void* lo = nullptr);

// sum_{v,d} (A[v][d] - (W Ht^T)[v][d])^2: Eq. 2 evaluated directly for dense A
// (FP32 products, FP64 sum of the squared residuals).  dpart: scratch of
// resid2_partials(V, D) doubles; the result is written to *out (host).
int64_t resid2_partials(int V, int D);
cudaError_t resid2_dense(const float* A, int64_t lda, const float* W, const float* Ht, int V, int D, int K, int Kp,
                         double* dpart, double* out, cudaStream_t s);

// S (Kp x Kp) = X^T X for X (N x Kp): split-N partials, FP64 fixed-order sum.
struct GramWork {
  float* d_part = nullptr;   // n_chunks x Kp x Kp
  int n_chunks = 0, chunk = 0, N = 0, Kp = 0;
  int groups = 1, tpg = 0;   // upper-triangle tile groups (gram_tri_kernel)
};
cudaError_t gram_setup(GramWork& g, int N, int Kp);
void gram_free(GramWork& g);
// skip_count (gram_tri_kernel shapes only): when *skip_count >= skip_need
// the chunk partials are taken as already formed (by the W update's workers,
// in this kernel's order) and only the reduction runs.
cudaError_t gram_run(const GramWork& g, const float* X, float* S, int K, cudaStream_t s,
                     const int* skip_count = nullptr, int skip_need = 0);
// The chunked Gram applies (gram_tri_kernel with one tile group): the shapes
// for which the W update's workers can form the partials.
bool gram_tri_single_group(const GramWork& g);
// Re-chunk a GramWork (chunk rows per partial, n_chunks <= the chunks its
// buffer was set up for); the tile grouping follows.
void gram_rechunk(GramWork& g, int chunk, int n_chunks);
// S (K x K) = X^T X for X (N x K, row stride ldx) with caller-provided
// partial storage: n_chunks * K * K floats, chunk rows per partial.
cudaError_t gram_run_scratch(const float* X, int N, int K, int64_t ldx, float* part, int n_chunks, int chunk,
                             float* S, cudaStream_t s);
// Same result through the tensor cores (3xTF32, split-N partials).
cudaError_t gram_setup_tc(GramWork& g, int N, int Kp);
cudaError_t gram_run_tc(const GramWork& g, const float* X, float* S, int K, int* d_status, cudaStream_t s,
                        bool bf16 = false);

// ---------------------------------------------------------------------------
// Tall-factor update (Alg. 2 regrouped): phase 1 GEMM, per-tile chain, phase 3.
// ---------------------------------------------------------------------------
struct ChainConfig {
  int cluster = 16;       // CTAs cooperating on the normalised chain
  int threads = 256;
  int rpt = 1;            // rows per thread
  int tt = 16;            // widest tile the configuration was sized for
};
constexpr int kMaxChainTile = 16;

// Y (N x Kp): base of tile [lo, hi) (see w_prep_run); X: factor (old on
// entry, tile columns new on exit); G: Gram.  prev_lo >= 0: the base still
// lacks the contribution of the new columns [prev_lo, lo) of X, which the
// kernel adds first.
cudaError_t chain_run(float* Y, float* X, const float* G, int N, int Kp, int lo, int hi, int prev_lo,
                      float eps, bool normalize, const ChainConfig& cfg, int* d_status,
                      cudaStream_t s);
bool chain_config_for(int N, bool normalize, int T, ChainConfig* cfg);
bool chain_config_cluster(int N, int T, int cl, ChainConfig* cfg);

// Whole H update in one launch (rows independent): X (N x Kp) old -> new in
// place, B = R, G = S.  skip (device int, optional): when nonzero at launch
// the kernel leaves X as it is (the converged part of a sweep loop).
// pack_rows: two rows per lane group at every row count (fewer CTAs and
// shared-memory loads for the same arithmetic; for problems that share the
// GPU with others, as batch members do).
cudaError_t h_update_run(float* X, const float* B, const float* G, int N, int K, int Kp, float eps,
                         int* status, cudaStream_t s, const int* skip = nullptr, bool pack_rows = false);
// The same update with the off-tile sums on the tensor cores (3xTF32 with
// per-plane compensated folds); supported for 16 <= Kp <= 512.
bool h_update_tc_supported(int Kp);
cudaError_t h_update_tc_run(float* X, const float* B, const float* G, int N, int K, int Kp, float eps,
                            int* status, cudaStream_t s);
// Base of W tile [lo, lo + T) (T <= 16) for the chain: Y[:, tile] from B = P,
// G = Q and the current (partly updated) factor X, with the new columns
// [0, new_end).
// B == nullptr leaves the data term out; then, with Ylo (N x 16) given, the
// compensated sum is returned unrounded as Y[:, tile] + Ylo (the caller adds
// P to Y first: the two cancel, so the early rounding would be magnified).
// With co given (B == nullptr, lo = new_end = 0, T = 16), the sum and its
// compensation go to co->base and co->comp in the W chain's register order
// instead of Y and Ylo.
struct ChainOrder;
cudaError_t w_prep_run(const float* X, const float* B, const float* G, float* Y, int N, int K, int Kp, int lo,
                       int new_end, int* status, cudaStream_t s, int T, float* Ylo = nullptr,
                       const ChainOrder* co = nullptr);
constexpr int kRowTile = 16;   // tile width of the row-parallel update kernels

// The register order of the persistent W update's column chain for one
// 16-column tile: the 16-byte quad of row v, tile columns 4 q .. 4 q + 3,
// is quad ((c * rpt + i) * 4 + q) * kChainRowThreads + r of the buffer, with
// chain CTA c = v / chain_rows, register row i and row thread r from
// v - c * chain_rows = i * kChainRowThreads + r.  A chain row thread loads
// its rows of a tile with rpt x 4 loads of a warp's 512 consecutive bytes.
constexpr int kChainRowThreads = 480;
struct ChainOrder {
  float* base = nullptr;       // tile 0's early base less P
  float* comp = nullptr;       // its compensation
  int chain_rows = 0;
  int rpt = 0;
};
__host__ __device__ __forceinline__ long long chain_quad(int v, int q, int chain_rows, int rpt) {
  const int c = v / chain_rows, li = v - c * chain_rows;
  const int i = li / kChainRowThreads, r = li - i * kChainRowThreads;
  return (((long long)c * rpt + i) * 4 + q) * kChainRowThreads + r;
}

// Alg. 1 as written (no column tiling): the H and W updates column by
// column, K (H) or 2K (W) dependent grid-wide launches; `part` holds
// alg1_parts(V) floats (per-CTA sums of squares); `launches` (optional) is
// incremented by the number of kernels enqueued.
int alg1_parts(int V);
cudaError_t alg1_update_h(float* Ht, const float* R, const float* S, int D, int K, int Kp, float eps,
                          cudaStream_t s, int* launches);
cudaError_t alg1_update_w(float* W, const float* P, const float* Q, int V, int K, int Kp, float eps, float* part,
                          int* status, cudaStream_t s, int* launches);

// Multiplicative update of the tall factor X (N x Kp): X <- X * B / (X G + delta)
// for the K valid columns (G symmetric K x K Gram); scratch: N x Kp.
cudaError_t mu_update(float* X, const float* B, const float* G, float* scratch, int N, int K, int Kp, float delta,
                      cudaStream_t s, int* launches);

// Whole W update in one launch: cluster 0 runs the column chain over all
// tiles, the other clusters compute the tile bases (blocks the chain finds
// unclaimed it computes itself, so the result does not depend on how many
// clusters are resident at once).
struct WPersistConfig {
  int cluster = 16;       // chain CTAs (one cluster)
  int rpt = 1;
  int n_workers = 0;      // worker CTAs (one per SM outside the chain)
  int worker_rows = 128;
  int worker_wr = 1;      // rows per worker lane group (2 for Kp >= 128)
  int chain_rows = 0;     // rows per chain CTA
  int stage_rows = 128;   // rows a worker stages at once (its whole block where it fits)
  size_t chain_smem = 0;
  size_t worker_smem = 0;
  bool tc = false;        // the workers form the tile bases on the tensor cores
  // The worker grid launched in plain stream order, after the chain grid has
  // finished (as a tool that serialises launches runs the two): the chain
  // then forms every tile base itself.  Default: a programmatic dependent.
  bool workers_after_chain = false;
};
// tc: the workers form the tile bases on the tensor cores (TF32 pairs).
bool w_persistent_config(int N, int Kp, WPersistConfig* cfg, bool tc = false);
// d_sync: w_sync_ints(K) ints (zeroed by the call, on the stream).
size_t w_sync_ints(int K);
// pre0 != nullptr: w_chain_order(Yc, ...) slot 0 plus its compensation
// (pre0 = the order's comp) already hold tile 0's base less P (w_prep_run
// with B = nullptr, lo = new_end = 0 and that ChainOrder); the launch then
// adds P there.
// wait_ns: limit of every device wait (0: kWaitLimitNs); extra_arrivals > 0
// makes the workers wait for more chain arrivals than exist (tests of the
// timeout path: the waits run out, ST_TIMEOUT is set and the chain computes
// the remaining bases itself).
// spart != nullptr (SIMT workers, Kp <= 256): the workers also form the Gram
// partials of the new factor for the row chunks of w_persistent_blocks (chunk
// w = worker w's rows, Kp x Kp each, upper triangle), in gram_tri_kernel's
// order for those chunks, and count the finished block columns at
// d_sync[w_sync_sdone_offset(K)] (nb x ceil(K / 16) when all are done).
// Yc: w_chain_base_floats() floats of scratch (two slots of tile bases in
// the chain's register order, then tile 0's early-base compensation).
// after_chain (optional) is recorded right after the chain grid's launch:
// work that waits for it sees the whole new factor (every store of the chain
// precedes its grid's end) while the worker grid may still be forming S's
// last block columns.  (Within a stream capture the record adds no node, so
// the worker grid stays the chain grid's programmatic dependent.)
size_t w_chain_base_floats();
// Tile 0's early base and its compensation in the chain's order (for
// w_prep_run) within Yc for this configuration.
ChainOrder w_chain_order(float* Yc, int N, const WPersistConfig& cfg);
cudaError_t w_persistent_run(float* X, const float* P, const float* Q, float* Yc, int N, int K, int Kp,
                             float eps, int* d_sync, int* d_status, const WPersistConfig& cfg, cudaStream_t s,
                             const float* pre0 = nullptr, unsigned long long wait_ns = 0, int extra_arrivals = 0,
                             float* spart = nullptr, cudaEvent_t after_chain = nullptr);
// Row blocks of the two-grid W update: nb blocks of per rows (the last
// shorter), one per worker CTA.
void w_persistent_blocks(int N, const WPersistConfig& cfg, int* nb, int* per);
size_t w_sync_sdone_offset(int K);

// ---------------------------------------------------------------------------
// Misc kernels.
// ---------------------------------------------------------------------------
// Element (r, c < cols) of a rows x ld buffer = SplitMix64 draw r*cols + c
// (or c*rows + r for the transposed variant); padding columns are zeroed.
cudaError_t fill_uniform_splitmix(float* dst, int rows, int cols, int ld, uint64_t seed,
                                  cudaStream_t s);
cudaError_t fill_uniform_splitmix_t(float* dst, int rows, int cols, int ld, uint64_t seed,
                                    cudaStream_t s);
cudaError_t normalize_columns(float* X, int N, int K, int ld, cudaStream_t s);
// dst (rows x ld, BF16, round to nearest) = src (rows x cols, row stride ld), pads zero.
// dst (rows x ldd, BF16 round-to-nearest-even) = src (rows x cols, row stride lds); columns cols..ldd zero.
cudaError_t convert_bf16(const float* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                         cudaStream_t s, void* lo = nullptr);
// frob2 = normA2 - 2 <W, P> + <S, Q>, appended to the history ring.  The
// dot products use compensated FP32 arithmetic (Dot2) per thread and FP64
// across threads; `partial` holds 2 * n_partial doubles.
cudaError_t objective_run(const float* W, const float* P, int V, int Kp, const float* S,
                          const float* Q, double normA2, double* partial, int n_partial,
                          double* out, unsigned* d_counter, int hist_cap, cudaStream_t s);
// The two halves of objective_run, for callers that overlap <W, P> (needs the
// new W and P only) with the Gram S: partials of <W, P> (partial[0..n)), then
// the <S, Q> partials (partial[n..n + 64)) and the history entry.  partial
// holds at least n + 64 doubles.  `last` (optional, device) receives the
// new history entry as well.
cudaError_t objective_wp(const float* W, const float* P, int V, int Kp, double* partial, int n_partial,
                         cudaStream_t s);
cudaError_t objective_finish(int Kp, const float* S, const float* Q, double normA2, double* partial,
                             int n_partial, double* out, unsigned* d_counter, int hist_cap, cudaStream_t s,
                             double* last = nullptr);
constexpr int kSumsqBlocks = 592;
cudaError_t sumsq_dense_f64(const float* A, int64_t rows, int64_t cols, int64_t ld,
                            double* d_out, int* d_bad, cudaStream_t s);
cudaError_t transpose_f32(const float* src, int rows, int cols, int lds, float* dst, int ldd,
                          cudaStream_t s);

// ---------------------------------------------------------------------------
// Warm start (warmstart.cu).
// ---------------------------------------------------------------------------
cudaError_t scale_shift(float* x, int64_t n, float a, float b, cudaStream_t s);
// h_out[0] = sum (H - Href)^2, h_out[1] = sum Href^2 (sum H^2 without Href),
// over rows x K of row-stride-ld buffers; FP64; synchronises the stream.
// d_part holds diff_norm_partials() doubles.
cudaError_t diff_norm(const float* H, const float* Href, int rows, int K, int ld, double* d_part, double* h_out,
                      cudaStream_t s);
size_t diff_norm_partials();
// One sweep's check on the device, for sweep loops that read back only every
// few sweeps: state[0] = done, state[1] = sweeps run.  Unless done, the
// relative change sqrt(sum (H - Href)^2 / sum Href^2) (sqrt(sum H^2) when the
// second sum is zero; Href null: H^2) is formed in FP64 from the partials of
// d_part, written to trace[sweep - 1], state[1] = sweep, and state[0] = 1
// when it is <= tol.  copy_unless_done copies n floats unless state[0].
cudaError_t diff_check(const float* H, const float* Href, int rows, int K, int ld, double* d_part, float tol,
                       int sweep, double* trace, int* state, cudaStream_t s);
cudaError_t copy_unless_done(float* dst, const float* src, int64_t n, const int* state, cudaStream_t s);
// The check of diff_check from nblk (sum, sum) partial pairs already formed.
cudaError_t sweep_check(const double* d_part, int nblk, float tol, int sweep, double* trace, int* state,
                        cudaStream_t s);
// One sweep of a fixed-W H loop (nmf_warm_h): the H update of X in place,
// skipped once state[0] is set, with the change against Href (or, Href null,
// against the values it replaces) summed in the update's own write-back into
// part (h_sweep_partials(N) doubles), then the check of diff_check.  Hprev
// (N x Kp) is scratch for the row-per-warp form (Kp <= 32) without Href.
size_t h_sweep_partials(int N);
cudaError_t h_update_sweep(float* X, const float* B, const float* G, int N, int K, int Kp, float eps, int* status,
                           cudaStream_t s, const float* Href, float* Hprev, double* part, float tol, int sweep,
                           double* trace, int* state);
// Network forward of `rows` inputs x (row stride ldx) into y (row stride ldy).
cudaError_t mlp_forward_dev(nmf_mlp* n, const float* x, int64_t ldx, int rows, float* y, int64_t ldy,
                            cudaStream_t s);
int mlp_K(const nmf_mlp* n);

}  // namespace plnmf
