/*
 * nmf.h — C ABI of the B300 FAST-HALS / PL-NMF library (libplnmf.so).
 *
 * The library factorises a non-negative matrix A (V x D) as A ~= W H with
 * W (V x K) and H (K x D) non-negative, minimising 1/2 ||A - WH||_F^2
 * (Sec. 1, Eq. 1; Sec. 2.1, Eq. 2) with the FAST-HALS iteration of Alg. 1,
 * whose column-sequential factor updates are regrouped into column tiles as in
 * Alg. 2 (Sec. 3.3, Eqs. 4-6).  All compute runs in CUDA kernels on one GPU.
 *
 * Conventions for every entry point
 *   - Pointers marked "device" must be device (or managed) memory of the
 *     current CUDA device; pointers marked "host or device" may be either
 *     (the copy direction is inferred through unified addressing).
 *   - Matrices are row-major with the stated shapes.
 *   - Every call returns an nmf_status and never aborts or traps.  A CUDA
 *     error raised asynchronously by an earlier launch is reported by the
 *     next call that synchronises (NMF_ECUDA).
 *   - A context is bound to one CUDA stream and is not thread-safe; use one
 *     context per stream/thread.
 */
#ifndef PLNMF_NMF_H
#define PLNMF_NMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NMF_OK = 0,
  NMF_EINVAL = 1,       /* bad argument (shape, pointer, negative or non-finite A, ...) */
  NMF_ENOMEM = 2,       /* device allocation failed */
  NMF_ECUDA = 3,        /* a CUDA call or kernel failed */
  NMF_ETIMEOUT = 4,     /* a bounded device-side wait expired (status word set by a kernel) */
  NMF_ENUMERIC = 5,     /* a column norm was zero or not finite */
  NMF_EBUSY = 6,        /* context is being captured or used by another call */
  NMF_EUNSUPPORTED = 7  /* valid request this build does not implement (shape limits) */
} nmf_status;

typedef enum { NMF_DENSE_F32 = 0, NMF_CSR_F32_I32 = 1 } nmf_format;
typedef enum { NMF_PREC_FP32 = 0, NMF_PREC_BF16 = 1 } nmf_precision;

/*
 * Problem description (Sec. 1: A in R+^{V x D}, rank K; Alg. 1 inputs A, eps
 * and a random non-negative initialisation).
 *   V, D, K      1 <= K <= min(V, D); K <= 512 in this build.
 *   fmt          NMF_DENSE_F32: `dense` (device, V x D row-major, leading
 *                dimension `ld` >= D).
 *                NMF_CSR_F32_I32: `row_ptr` (V+1), `col_idx` (nnz), `val`
 *                (nnz), device, rows = words (V), columns = documents (D);
 *                row_ptr[0] = 0, non-decreasing, column indices in [0, D).
 *                The caller owns A; it must stay valid and unchanged for the
 *                life of the context.
 *   W0, H0       optional initial factors (host or device), W0 V x K and
 *                H0 K x D row-major.  NULL -> U[0,1) from `seed` drawn with
 *                the SplitMix64 stream defined in the Python module
 *                paper_1904_07935_b300.synth (entry r*cols+c of stream
 *                seed ^ 0x5757.. for W, seed ^ 0x4848.. for H).  Either way
 *                the columns of W are then scaled to unit L2 norm.
 *   eps          clamp floor of Alg. 1 (paper leaves it unset; 0 -> 1e-16).
 *   tile_T       column-tile width T of Alg. 2; 0 -> library choice (16, the
 *                register tile of the column chain).  Honoured (1..16) for the
 *                W update when flags has NMF_FLAG_MULTI_LAUNCH_W (per-tile
 *                launches); otherwise any value means the library choice.
 *                nmf_query reports the width in use.
 *   prec         NMF_PREC_FP32 (all FP32) or NMF_PREC_BF16 (dense A only:
 *                products A H^T, A^T W and the Gram matrices on the tensor
 *                cores with BF16 operands and FP32 accumulation; column
 *                updates and norms FP32; A is copied once to a BF16 pair
 *                A_hi + A_lo, see NMF_FLAG_BF16_SINGLE_A).
 *   stream       cudaStream_t to run on (NULL -> the context creates one).
 */
typedef struct {
  int32_t V, D, K;
  int32_t fmt;
  const float* dense;
  int64_t ld;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const float* val;
  int64_t nnz;
  const float* W0;
  const float* H0;
  uint64_t seed;
  float eps;
  int32_t tile_T;
  int32_t prec;
  void* stream;
  int32_t flags;        /* NMF_FLAG_* bits, 0 for the defaults */
} nmf_problem;

/* nmf_problem.flags.  The FP32 path computes its Gram matrices on the SIMT
 * FP32 pipes by default: the tensor cores accumulate in FP32 with
 * truncation, which loses ~K * 2^-24 relative accuracy in a K-term sum, too
 * much for the H update on the first iterations from a random start (it
 * cancels S h ~ 60 against h + R).  NMF_FLAG_TC_GRAMS moves the FP32 Grams
 * to the tensor cores (3xTF32) anyway.  The BF16 precision form always uses
 * the tensor cores. */
#define NMF_FLAG_TC_GRAMS 1
/* Run the W update as separate launches per column tile instead of one launch
 * holding the column chain and the tile-base workers (the default wherever a
 * chain cluster of 16 or 8 CTAs and at least one worker cluster fit). */
#define NMF_FLAG_MULTI_LAUNCH_W 2
/* BF16 form (NMF_PREC_BF16): take the dense products A^T W and A H^T through
 * the SIMT-staged tensor-core kernel instead of the TMA-fed one (the default
 * where the driver exposes tensor-map encoding).  That kernel rounds A to BF16
 * once (as NMF_FLAG_BF16_SINGLE_A). */
#define NMF_FLAG_NO_TMA 4
/* BF16 form, operand precision.  By default every tensor-core operand is
 * carried as a BF16 pair, X = X_hi + X_lo with X_hi = bf16(X) and
 * X_lo = bf16(X - X_hi) (about 16 significant bits): the products use
 * A_hi F_hi + A_lo F_hi + A_hi F_lo and the Grams F_hi F_hi + F_lo F_hi +
 * F_hi F_lo, three BF16 MMAs per tile with FP32 accumulation (F = the factor
 * operand).  NMF_FLAG_BF16_SINGLE_FACTORS rounds the factor operands to BF16
 * once (two MMAs per product tile, one per Gram tile); NMF_FLAG_BF16_SINGLE_A
 * rounds A once as well (one MMA per tile; the fit is then to bf16(A), whose
 * error is about 2^-9 / sqrt(3) of A). */
#define NMF_FLAG_BF16_SINGLE_A 8
#define NMF_FLAG_BF16_SINGLE_FACTORS 16
/* Form the factor updates' off-tile sums (Eqs. 4 and 6: new columns left of
 * each tile, old columns right of it) on the tensor cores, in the H update
 * and in the W update's tile bases: both operands split into TF32 pairs
 * (hi + lo, three kind::tf32 MMAs per K step, about 2^-21 relative per
 * product), each 32-column plane accumulated on its own and the planes' sums
 * folded with compensation.  The in-tile column chains stay on the CUDA
 * cores. */
#define NMF_FLAG_TC_UPDATES 32

typedef struct nmf_ctx nmf_ctx;

/* Validates the problem (shapes, CSR structure, A >= 0 and finite, A not
 * identically zero: the relative error is defined only for ||A|| > 0), builds
 * the transposed CSR of A and the SpMM work plans, computes ||A||_F^2 in
 * FP64, allocates W, H and all intermediates and initialises the factors.
 * On success *out owns every device buffer it allocated.  Synchronous. */
nmf_status nmf_init(const nmf_problem* p, nmf_ctx** out);

/* Runs n_iters iterations of Alg. 1 (H update, then W update) on the
 * context's stream, asynchronously.  Each iteration also records the
 * objective (Eq. 2 times 2, via the trace identity, FP64) of the new
 * factors.  The first call captures the iteration in a CUDA graph. */
nmf_status nmf_iterate(nmf_ctx* c, int32_t n_iters);

/* Synchronises the stream and returns the latest objective
 * frob2 = ||A - WH||_F^2 and rel = sqrt(frob2 / ||A||_F^2) (Sec. 6.2.2).
 * For dense A the value is Eq. 2 evaluated directly for the current factors,
 * sum of (A - WH)^2 with FP32 products and FP64 accumulation (no cancellation;
 * in the BF16 form it measures the fit to the FP32 A, not to its BF16 copy).
 * For CSR A it is the latest per-iteration value (trace identity).
 * Before any iteration it evaluates the initial factors.  Also reports
 * device-side status (NMF_ETIMEOUT / NMF_ENUMERIC) raised since the last
 * call.  Either output pointer may be NULL. */
nmf_status nmf_error(nmf_ctx* c, double* frob2, double* rel);

/* Copies the n most recent per-iteration objectives (oldest first) to host
 * memory `out` (FP64).  n <= number of iterations run and <= 4096. */
nmf_status nmf_objective_history(nmf_ctx* c, double* out, int32_t n);

/* W: V x K, H: K x D, row-major FP32, host or device.  Either may be NULL.
 * Synchronous. */
nmf_status nmf_get_factors(nmf_ctx* c, float* W, float* H);
/* Replaces the factors (checkpoint / resume).  W is used as given (no
 * normalisation).  Synchronous. */
nmf_status nmf_set_factors(nmf_ctx* c, const float* W, const float* H);

/* One iteration (Alg. 1, factor updates in the order of Alg. 2) on factors
 * held by the caller: the same as nmf_set_factors(W_in, H_in),
 * nmf_iterate(1), nmf_error(frob2), nmf_get_factors(W_out, H_out), with the
 * copies overlapped with the iteration.
 *   W_in, W_out  V x K, H_in, H_out  K x D, row-major FP32; any may be NULL
 *                (that factor is neither loaded nor returned).  W_in may
 *                equal W_out and H_in H_out (each input is read before its
 *                output is written).  W_in is used as given (no
 *                normalisation).
 *   frob2        NULL or the objective ||A - W H||_F^2 after the iteration
 *                (as nmf_error reports it).
 * When every buffer given is pinned host memory (cudaHostAlloc,
 * cudaHostRegister) or device memory, the copies and the iteration run as one
 * CUDA graph (captured on the first call, reused while the pointers stay the
 * same): H_in is copied while R = A^T W and S = W^T W of the new W run, H_out
 * while P, Q and the W update run, W_out beside the objective.  R of the new
 * W is not formed (a following nmf_iterate forms it).  Other host memory is
 * copied before and after, without overlap.  Synchronous; returns the
 * iteration's device status like nmf_error. */
nmf_status nmf_iterate_host(nmf_ctx* c, const float* W_in, const float* H_in, float* W_out, float* H_out,
                            double* frob2);

/* Individual steps of one iteration, for per-step parity and timing
 * (the steps of Alg. 1; all asynchronous on the context stream):
 *   NMF_STEP_R        R = A^T W
 *   NMF_STEP_S        S = W^T W
 *   NMF_STEP_UPDATE_H H update with R, S           (Alg. 2 order)
 *   NMF_STEP_P        P = A H^T
 *   NMF_STEP_Q        Q = H H^T
 *   NMF_STEP_UPDATE_W W update with P, Q           (Alg. 2 order)
 *   NMF_STEP_OBJECTIVE objective of current W, H using the current P and the
 *                     Gram of the current W (recomputed) and Q. */
typedef enum {
  NMF_STEP_R = 0, NMF_STEP_S = 1, NMF_STEP_UPDATE_H = 2, NMF_STEP_P = 3,
  NMF_STEP_Q = 4, NMF_STEP_UPDATE_W = 5, NMF_STEP_OBJECTIVE = 6
} nmf_step;
nmf_status nmf_run_step(nmf_ctx* c, int32_t step);

/* Internal buffers, exposed for per-step parity tests (row-major FP32):
 *   NMF_BUF_W  V x K        NMF_BUF_HT D x K (H transposed)
 *   NMF_BUF_R  D x K        NMF_BUF_P  V x K
 *   NMF_BUF_S  K x K        NMF_BUF_Q  K x K
 * `count` must equal the element count of the buffer.  dst/src host or
 * device.  Synchronous. */
typedef enum {
  NMF_BUF_W = 0, NMF_BUF_HT = 1, NMF_BUF_R = 2, NMF_BUF_P = 3, NMF_BUF_S = 4, NMF_BUF_Q = 5
} nmf_buffer;
nmf_status nmf_get_buffer(nmf_ctx* c, int32_t which, float* dst, int64_t count);
nmf_status nmf_set_buffer(nmf_ctx* c, int32_t which, const float* src, int64_t count);

/* Alg. 1 as written, without the column tiling (the form the paper's
 * regrouping, Alg. 2, is measured against; Sec. 5, Table 5): the same
 * products (R = A^T W, P = A H^T, Q = H H^T, S = W^T W) and objective, but
 * the H and W updates run column by column, each column one grid-wide step
 * (W: two, the second normalising the column before the next one reads it),
 * so an iteration is 3K + O(1) dependent launches.  H^T S_k and W Q_k use
 * the current factor and include the j = k term (Alg. 1's H and W loops);
 * FP32 with FP32 dot products (no compensation).  n_iters iterations of
 * the context's factors (same entry/exit state as nmf_iterate, so the two
 * can be mixed).  step_ms: NULL -> the iterations run as a CUDA graph
 * (captured on the first call), asynchronous on the context stream; else
 * NMF_PROFILE_STEPS floats receive the mean milliseconds of each step as
 * in nmf_profile (eager launches, CUDA events), synchronous.  Returns
 * NMF_EINVAL for n_iters < 0 or a NULL context. */
nmf_status nmf_iterate_alg1(nmf_ctx* c, int32_t n_iters, float* step_ms);

/* Multiplicative updates (Lee & Seung 2001; the simplest NMF algorithm, the
 * paper's comparison baseline, Sec. 2): H <- H * (W^T A) / (W^T W H + eps),
 * then W <- W * (A H^T) / (W H H^T + eps), elementwise, W not normalised;
 * the same products, Grams and objective as nmf_iterate.  Arguments, state
 * and step_ms as nmf_iterate_alg1. */
nmf_status nmf_iterate_mu(nmf_ctx* c, int32_t n_iters, float* step_ms);

/* Step timing (tracing): runs n_iters iterations eagerly (no graph) with a
 * CUDA event between consecutive steps on the context stream and writes the
 * mean milliseconds per iteration of each step to step_ms[0..6]:
 *   0 R = A^T W, 1 H update, 2 P = A H^T, 3 Q = H H^T, 4 W update,
 *   5 S = W^T W of the new W, 6 objective.
 * The factors advance by n_iters iterations.  Synchronous. */
#define NMF_PROFILE_STEPS 7
nmf_status nmf_profile(nmf_ctx* c, int32_t n_iters, float* step_ms);

/* Introspection: tile width in use, cluster size of the W column chain,
 * number of kernel launches one iteration makes in the form run last
 * (nmf_iterate, nmf_iterate_alg1 or nmf_iterate_mu; before any of them, the
 * nmf_iterate form's count once its graph exists, else 0). */
nmf_status nmf_query(nmf_ctx* c, int32_t* tile_T, int32_t* chain_ctas, int32_t* launches_per_iter);

/* How the context runs the W side of an iteration (any output may be NULL):
 *   w_single_launch  1: the whole W update is one pair of launches (a
 *                    column-chain cluster and, as its programmatic
 *                    dependent, a grid of base-forming worker CTAs), 0:
 *                    per-tile launches.
 *   s_in_w_update    1: within nmf_iterate / nmf_profile those worker CTAs
 *                    also form the row-chunk partials of
 *                    S = W^T W of the new W (in the Gram kernel's order), so
 *                    the S step that follows only reduces them.
 *   s_chunks         the number of those row-chunk partials (0 if none). */
nmf_status nmf_query_form(nmf_ctx* c, int32_t* w_single_launch, int32_t* s_in_w_update, int32_t* s_chunks);

/* Limits of the W update's device-side waits (the two-grid form that
 * replaces Alg. 3's two host synchronisations per column with hand-offs
 * between the column chain and the CTAs forming the tile bases).
 *   wait_ns          limit of every such wait in nanoseconds; 0 restores the
 *                    library default (200 ms).
 *   extra_arrivals   0 in normal use.  A positive value makes the base-forming
 *                    CTAs wait for that many more chain arrivals than will
 *                    ever come, so that their waits run out: a way to test the
 *                    failure path without a GPU fault.  Their waits then set
 *                    the status word (the next nmf_error / nmf_get_factors
 *                    returns NMF_ETIMEOUT once), and the chain computes the
 *                    bases they left, so the factors stay those of a normal
 *                    update.
 * Takes effect at the next nmf_iterate (the iteration graph is re-captured).
 * NMF_EINVAL for wait_ns < 0 or extra_arrivals < 0; NMF_EUNSUPPORTED when the
 * context runs the per-tile W launches, which have no such waits. */
nmf_status nmf_set_wait_limits(nmf_ctx* c, int64_t wait_ns, int32_t extra_arrivals);

/* Work schedule of the two sparse products of Alg. 1, P = A H^T (over the
 * CSR rows of A) and R = A^T W (over those of A^T), for CSR contexts (the
 * library CSR products of Sec. 4.2).  A row with more than seg non-zeros is
 * cut into seg-long pieces that separate warps gather; the piece that
 * finishes last adds the pieces' partial rows in piece order, so a product
 * is bit-reproducible for a given seg, while another seg changes the
 * rounding of long rows' sums (the words of the Zipf head, and long
 * documents).  Default 512 for both.
 * nmf_set_spmm_split: seg_P and seg_R >= 16, or 0 for no split (one piece per
 *   row).  NMF_EINVAL for other values.
 * nmf_tune_spmm: times each product with seg in {128, 256, 512, 1024, no
 *   split} (CUDA events on the context stream, one warm-up and three timed
 *   runs each, the current factors) and keeps the fastest; seg_P / seg_R
 *   (may be NULL) return the choices (0: no split).  P's buffer is
 *   overwritten (it is recomputed by every iteration) and R is recomputed for
 *   the current W.  The choice depends on the timings, so two contexts tuned
 *   separately can choose differently; nmf_set_spmm_split with the returned
 *   values reproduces a tuned context's schedule exactly.
 * Both: synchronous; NMF_EUNSUPPORTED for dense A; take effect at the next
 * nmf_iterate (the iteration graph is re-captured).  Not while the context is
 * a member of a batch (destroy the batch first). */
nmf_status nmf_set_spmm_split(nmf_ctx* c, int32_t seg_P, int32_t seg_R);
nmf_status nmf_tune_spmm(nmf_ctx* c, int32_t* seg_P, int32_t* seg_R);

/* Launch order of the two grids of the W update (contexts that run it as
 * the column-chain cluster grid plus the tile-base worker grid, the form that
 * replaces Alg. 3's two host synchronisations per column, Sec. 4.2):
 *   on = 0  default: the worker grid is a programmatic dependent of the chain
 *           grid and forms the tile bases while the chain runs;
 *   on = 1  the worker grid starts only after the chain grid has finished, as
 *           a tool that serialises kernel launches runs the two.  The chain
 *           then claims and forms every tile base itself (after waiting
 *           50 us per tile for workers that never come); the workers find
 *           every base formed and only form the Gram partials of the new W.
 *           The factors and the objective are bit-identical to on = 0, the W
 *           update is slower.  For tests of that schedule.
 * Takes effect at the next nmf_iterate (the iteration graph is re-captured).
 * NMF_EINVAL for on not 0 or 1; NMF_EUNSUPPORTED when the context runs the
 * per-tile W launches. */
nmf_status nmf_set_w_workers_after_chain(nmf_ctx* c, int32_t on);

/* Dense product on the tensor cores (tcgen05), a library utility used by the
 * iteration and exposed for testing:  C (M x N) = op(A) (M x K) * B (K x N),
 * op(A) = A (row-major, lda) or A^T (A stored K x M row-major, lda) when
 * transA != 0; B row-major K x N (ldb); C row-major (ldc).  prec:
 * NMF_PREC_FP32 -> 3xTF32 split (near-FP32 accuracy), NMF_PREC_BF16 -> BF16
 * operands.  FP32 accumulation.  All pointers device; asynchronous on
 * `stream`.  Returns NMF_EINVAL for non-positive sizes or null pointers. */
nmf_status nmf_gemm(int32_t M, int32_t N, int32_t K, const float* A, int64_t lda, int32_t transA,
                    const float* B, int64_t ldb, float* C, int64_t ldc, int32_t prec, void* stream);

/* Batched form: many independent problems advanced together (repeated NMF
 * of many small matrices; the paper motivates repeated factorisation in
 * Sec. 1).  A batch holds existing contexts ("members"); one CUDA graph
 * holds one iteration of every member, each member's launches on its own
 * stream as parallel branches, so the GPU runs the members side by side.
 *
 * nmf_batch_create: members must be distinct contexts on distinct streams,
 *   and `stream` (the batch's launch stream; NULL = a new one owned by the
 *   batch) must differ from all of them (NMF_EINVAL otherwise, and for
 *   n < 1).  Members switch to the per-tile W launches (the two-grid W
 *   update holds every SM) and to H-update CTAs of two rows per lane group
 *   (fewer, fuller CTAs for SMs that the members share; the same
 *   arithmetic); a member's own single-problem graph is re-captured on its
 *   next nmf_iterate.  autotune != 0: for each member,
 *   timed with CUDA events from the same start: (1) sparse A: the SpMM
 *   schedule of each product, rows longer than seg non-zeros split into
 *   seg-long items (seg in 128, 256, 512, 1024) or no split, fastest of
 *   three runs; (2) the W update's column-tile width T (8, 12 or 16) and its
 *   column chain's cluster size (4, 8 or 16 CTAs, where the rows fit), least
 *   SM-time (chain CTAs x time of three updates).  W is restored, so tuning
 *   does not advance the factorisation.  Synchronous.  The batch does not
 *   own the members: destroy the batch before them.
 * nmf_batch_iterate: n_iters iterations of every member, asynchronous on the
 *   batch stream; ordered after all work already queued on the members'
 *   streams, and each member's stream is made to wait for the batch, so
 *   nmf_error / nmf_get_factors on a member see the result.
 * nmf_batch_query: member i's chain cluster size and, if autotuned, the
 *   measured W-update time (microseconds) of the chosen size.
 * nmf_batch_query_schedule: member i's W tile width and the SpMM split
 *   lengths of the products P = A H^T and R = A^T W (0 for dense A; 2^30:
 *   no row is split).
 * nmf_batch_submit: nmf_init of ps[0..n) (each ps[i].stream NULL or
 *   distinct), an autotuned batch, n_iters iterations; the contexts are
 *   returned in outs (caller destroys them); on failure none is returned.
 *   Returns once the iterations are queued. */
typedef struct nmf_batch nmf_batch;
nmf_status nmf_batch_create(nmf_ctx* const* ctxs, int32_t n, int32_t autotune, void* stream, nmf_batch** out);
nmf_status nmf_batch_iterate(nmf_batch* b, int32_t n_iters);
nmf_status nmf_batch_query(nmf_batch* b, int32_t i, int32_t* chain_ctas, float* w_update_us);
nmf_status nmf_batch_query_schedule(nmf_batch* b, int32_t i, int32_t* tile_T, int32_t* spmm_seg_P,
                                    int32_t* spmm_seg_R);
void nmf_batch_destroy(nmf_batch* b);
nmf_status nmf_batch_submit(const nmf_problem* ps, int32_t n, int32_t n_iters, nmf_ctx** outs);

/* Learned warm start for new documents with W fixed (fixed-W H subproblem).
 * With W fixed, repeating the H loop of Alg. 1 (S = W^T W) is
 * exact coordinate descent on min_{h >= eps} ||a - W h||^2 per document and
 * converges to the unique optimum h*.  A small network predicts a starting
 * h from r = W^T a so that fewer sweeps are needed.  The network (not in the
 * paper): K -> hidden -> hidden -> K,
 *   z1 = x W1 + b1, a1 = GELU(z1), z2 = a1 W2 + b2, a2 = GELU(z2),
 *   z3 = a2 W3 + b3, y = softplus(z3)
 * with GELU(x) = x Phi(x) (erf form), softplus(x) = log(1 + e^x), = x above
 * 20; parameters [W1, b1, W2, b2, W3, b3], Wl row-major n_in x n_out, FP32.
 * Products on the tensor cores with BF16 operands and FP32 accumulation;
 * master weights, Adam state and elementwise work FP32.
 *
 * nmf_mlp_create: K and hidden positive multiples of 8 (row strides of the
 *   BF16 operands), NMF_EINVAL otherwise; He-uniform weights
 *   U(-sqrt(6/n_in), sqrt(6/n_in)) from SplitMix64 draws of seed + layer,
 *   zero biases.  NMF_EUNSUPPORTED without tensor-map support.
 * nmf_mlp_set_params / nmf_mlp_get_params: six arrays (host or device),
 *   sizes K*hidden, hidden, hidden*hidden, hidden, hidden*K, K.  Synchronous.
 * nmf_mlp_forward: Y (rows x K) = network(X (rows x K)); X device, Y host or
 *   device; asynchronous on `stream`.
 * nmf_mlp_grads: gradients of the mean squared error mean((y - T)^2) over
 *   rows x K at the current parameters into grads[0..5] (host or device;
 *   NULL entries skipped) and the loss into *loss.  X host or device, T
 *   device.  Synchronous.
 * nmf_mlp_train_step: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias
 *   corrected) on that loss; X host or device, T device; asynchronous on
 *   `stream` unless loss is non-NULL (then it synchronises to return it).
 *
 * nmf_warm_h: new documents `new_docs` (CSR, V = fixedW's V word rows,
 *   D = N documents, K = fixedW's K) against the current W of `fixedW`:
 *   R = A_new^T W (SpMM), h0 = network(R) (mlp != NULL) or, cold, SplitMix
 *   U[0,1) draws as nmf_init draws H (seed = new_docs->seed); then sweeps of
 *   the H loop with S = W^T W fixed until the stopping value is <= tol or
 *   max_sweeps sweeps ran.  Stopping value: with H_ref (K x N row-major,
 *   host or device) ||H - H_ref||_F / ||H_ref||_F, else the relative change
 *   ||H_s - H_{s-1}||_F / ||H_{s-1}||_F.  Outputs: H_out (K x N row-major,
 *   host or device), R_out (N x K row-major, optional), *sweeps_out, and
 *   trace[s] = the stopping value after sweep s + 1 (optional, max_sweeps
 *   doubles).  The stopping value is formed on the device in the H update's
 *   write-back (FP32 squares, FP64 sums) and the host reads it back once per
 *   32 sweeps; sweeps after the one that met tol leave H as it is.  W and
 *   the context's own H are not changed.  Synchronous. */
typedef struct nmf_mlp nmf_mlp;
nmf_status nmf_mlp_create(int32_t K, int32_t hidden, uint64_t seed, nmf_mlp** out);
nmf_status nmf_mlp_set_params(nmf_mlp* n, const float* const* params);
nmf_status nmf_mlp_get_params(nmf_mlp* n, float* const* params);
nmf_status nmf_mlp_forward(nmf_mlp* n, const float* X, int32_t rows, float* Y, void* stream);
nmf_status nmf_mlp_grads(nmf_mlp* n, const float* X, const float* T, int32_t rows, float* const* grads,
                         double* loss);
nmf_status nmf_mlp_train_step(nmf_mlp* n, const float* X, const float* T, int32_t rows, float lr, double* loss,
                              void* stream);
void nmf_mlp_destroy(nmf_mlp* n);
nmf_status nmf_warm_h(nmf_ctx* fixedW, nmf_mlp* mlp, const nmf_problem* new_docs, float tol, int32_t max_sweeps,
                      const float* H_ref, float* H_out, float* R_out, int32_t* sweeps_out, double* trace);

/* BF16 product with TMA-fed tensor-core MMAs (the kernel of the BF16 form,
 * the products R and P of Alg. 1): C (M x N, FP32, row-major, ldc) = A B^T with
 * A row-major M x K (lda) and B row-major N x K (ldb): both operands K-major
 * bfloat16 (uint16 bit patterns), FP32 accumulation in tensor memory.  A and
 * B must start on 16-byte boundaries and lda, ldb be multiples of 8;
 * NMF_EINVAL otherwise and for non-positive sizes, short strides or null
 * pointers; NMF_EUNSUPPORTED where the driver exposes no tensor-map encoding.
 * All pointers device; asynchronous on `stream`. */
nmf_status nmf_gemm_bf16(int32_t M, int32_t N, int32_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                         int64_t ldb, float* C, int64_t ldc, void* stream);

/* Gram matrix without device allocation (this entry point has no
 * counterpart in the paper; it serves callers that cannot call cudaMalloc,
 * for example a process whose device memory is entirely reserved up front
 * by its own pool allocator, or code running where an allocation's implicit
 * synchronisation is not allowed).
 *   S (K x K, row-major, device) = X^T X for X (N x K, device, row stride
 *   ldx >= K), FP32 on the SIMT pipes over row chunks; the chunks' partial
 *   sums are combined in a fixed order, with compensated FP32 additions
 *   (TwoSum) for up to 256 chunks and in FP64 beyond; asynchronous on
 *   `stream`.
 * The partial sums use one file-scope device array of
 * NMF_NOALLOC_SCRATCH_FLOATS floats (16 MiB) that every GPU loading the
 * library holds until the process exits.  The first call on a device looks
 * the array's address up (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  No cudaMalloc/cudaFree or
 * allocating library routine is called.  Every call shares the array, so
 * calls that overlap on the GPU (different streams, or devices sharing the
 * address space) race and must be serialised by the caller; the partials are
 * fully rewritten by each call.
 * Errors: NMF_EINVAL for null pointers or bad sizes; NMF_EUNSUPPORTED when
 * K * K exceeds the array (K > 2048); NMF_ECUDA for a failed lookup or launch. */
#define NMF_NOALLOC_SCRATCH_FLOATS (4 * 1024 * 1024)
nmf_status nmf_gram_noalloc(const float* X, int32_t N, int32_t K, int64_t ldx, float* S, void* stream);

/* Frees every device buffer and the graph of the context.  NULL is a no-op. */
void nmf_destroy(nmf_ctx* c);

const char* nmf_status_str(int32_t s);

#ifdef __cplusplus
}
#endif

#endif /* PLNMF_NMF_H */
