// Host runtime and C ABI (include/nmf.h): problem validation, transposed CSR
// and SpMM plans, buffers, the per-iteration launch sequence (Alg. 1 with the
// factor updates regrouped as in Alg. 2) and its CUDA-graph capture.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cstdlib>

#include "internal.cuh"

using namespace plnmf;

struct nmf_ctx {
  int V = 0, D = 0, K = 0, Kp = 0, T = 16, fmt = 0, prec = 0;
  bool use_tc = false;      // FP32 Grams on the tensor cores (3xTF32)
  bool tc_updates = false;  // off-tile sums of the factor updates on the tensor cores
  bool bf16 = false;        // precision form: BF16 tensor-core products and Grams
  void* A_bf16 = nullptr;   // BF16 copy of dense A (V x lda)
  bool tma = false;         // BF16 products through the TMA-fed kernel
  void* Ab8 = nullptr;      // BF16 A, V x ld8D (row stride a multiple of 8)
  void* ATb8 = nullptr;     // BF16 A^T, D x ld8V
  void* Ab8lo = nullptr;    // split form: bf16(A - Ab8), same layout (null: A rounded once)
  void* ATb8lo = nullptr;   // split form: bf16(A^T - ATb8)
  void* Fb8 = nullptr;      // BF16 transposed factor, Kp x max(ld8V, ld8D)
  void* Fb8lo = nullptr;    // split factor: bf16(factor - Fb8), same layout (null: factor rounded once)
  int64_t ld8V = 0, ld8D = 0;
  float* gpart = nullptr;   // BF16 form: split-K partial Grams, gsplits x Kp x Kp
  float* ppart = nullptr;   // dense FP32 products: split-K partials
  int splitR = 1, splitP = 1;
  int gsplits = 0;
  double* resid_part = nullptr;     // dense A: partials of the direct objective
  float eps = 1e-16f;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;          // second stream for the W tile bases
  cudaStream_t side2 = nullptr;         // third stream: <W, P> of the objective beside S and R
  bool w_persistent = false;            // whole W update as the chain cluster grid + the worker grid
  WPersistConfig wp;
  // The two-grid W update's workers also form the chunk partials of
  // S = W^T W of the new W (gramW chunked by the workers' row blocks); the
  // Gram kernel after it only reduces them, or forms any the workers left.
  bool ws_gram = false;
  int ws_need = 0;                      // finished block columns when the workers formed all partials
  GramWork gramW0;                      // gramW's own chunking (restored when ws_gram is turned off)
  int* d_sync = nullptr;
  unsigned long long wait_ns = 0;       // limit of the W update's device waits (0: library default)
  int extra_arrivals = 0;               // tests of the timeout path: a hand-off count that cannot be reached
  bool w_workers_after_chain = false;   // W worker grid in plain stream order after the chain grid
  bool h_pack_rows = false;             // H update: two rows per lane group at any row count (batch members)
  std::vector<cudaEvent_t> ev;          // fork / join events of the W update
  // A (caller-owned) and its transpose (context-owned, CSR only).
  const float* dense = nullptr;
  int64_t lda = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const float* va = nullptr;
  int64_t nnz = 0;
  int* rpT = nullptr;
  int* ciT = nullptr;
  float* vaT = nullptr;
  SpmmPlan planA, planAt;
  std::vector<int> h_rp, h_rpT;   // host row pointers of A and A^T (re-planning by the batch autotuner)
  int segA = 512, segAt = 512;    // SpMM schedule: rows longer than seg non-zeros split into seg-long items
  GramWork gramW, gramH;
  ChainConfig chainW, chainH;
  // Factors and intermediates, row stride Kp, padding columns kept at zero.
  float *W = nullptr, *Ht = nullptr, *R = nullptr, *P = nullptr, *S = nullptr, *Q = nullptr;
  float* Y = nullptr;       // phase-1 / phase-3 base, max(V, D) x Kp
  float* stage = nullptr;   // transpose staging, max(V, D) x Kp
  float* Yc = nullptr;      // tile bases in the chain's register order (persistent W update)
  double* obj_partial = nullptr;
  int n_obj_partial = 296;
  double* hist = nullptr;
  unsigned* d_counter = nullptr;
  int* d_status = nullptr;
  double normA2 = 0.0;
  bool s_valid = false;       // S == W^T W for the current W
  bool r_valid = false;       // R == A^T W for the current W
  cudaEvent_t evx[6] = {};    // fork / join events of the overlapped steps; [5]: the W chain grid done
  long long iters_run = 0;
  int launches_per_iter = 0;
  int launches_alg1 = 0, launches_mu = 0;   // per iteration of the comparator graphs
  int last_launches = 0;                    // per iteration of the form run last
  int launch_count = 0;       // kernels issued by the last enqueue sequence
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // Alg. 1 as written (nmf_iterate_alg1): per-CTA sums of squares, graph.
  float* alg1_part = nullptr;
  cudaGraph_t graph_alg1 = nullptr;
  cudaGraphExec_t graph_alg1_exec = nullptr;
  cudaGraph_t graph_mu = nullptr;           // nmf_iterate_mu
  cudaGraphExec_t graph_mu_exec = nullptr;
  // nmf_iterate_host: copies of host factors overlapped with the iteration.
  cudaStream_t side3 = nullptr;             // host copies beside the iteration
  cudaEvent_t evio[6] = {};
  cudaGraph_t graph_io = nullptr;
  cudaGraphExec_t graph_io_exec = nullptr;
  const void* io_key[5] = {};               // W_in, H_in, W_out, H_out, objective wanted
  double* d_obj_last = nullptr;             // objective of the last iteration (device)
  double* h_obj = nullptr;                  // its pinned host copy
  int* h_status = nullptr;                  // pinned copy of the status word after the iteration
};

namespace {

constexpr int kHistCap = 4096;

nmf_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return NMF_OK;
  if (e == cudaErrorMemoryAllocation) return NMF_ENOMEM;
  return NMF_ECUDA;
}

#define CK(x)                                  \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) return from_cuda(_e); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(count, 1));
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- launch sequence --------------------------------------------------------

// BF16 form with TMA: the factor operand of a product or Gram is the factor
// transposed to BF16 in Fb8 (W^T for R and S, H for P and Q); operand_ready
// means the iteration already made it for both branches.
cudaError_t bf16_operand(nmf_ctx* c, bool w, cudaStream_t s) {
  c->launch_count += 1;
  return w ? transpose_to_bf16(c->W, c->V, c->Kp, c->Kp, c->Fb8, c->ld8V, s, c->Fb8lo)
           : transpose_to_bf16(c->Ht, c->D, c->Kp, c->Kp, c->Fb8, c->ld8D, s, c->Fb8lo);
}

cudaError_t enq_product_R(nmf_ctx* c, cudaStream_t s = nullptr, bool operand_ready = false) {   // R = A^T W
  if (!s) s = c->stream;
  if (c->fmt == NMF_CSR_F32_I32) {
    c->launch_count += 1;
    return spmm_run(c->planAt, c->ciT, c->vaT, c->W, c->R, c->Kp, s);
  }
  GemmArgs a;
  a.M = c->D; a.N = c->Kp; a.Kin = c->V;
  a.A = c->dense; a.lda = c->lda; a.transA = 1;
  a.B = c->W; a.ldb = c->Kp;
  a.C = c->R; a.ldc = c->Kp;
  c->launch_count += 1;
  if (c->bf16 && c->tma) {
    // R (D x Kp) = A^T (D x V) * (W^T)^T with W^T (Kp x V) in BF16.
    if (!operand_ready) {
      cudaError_t e = bf16_operand(c, true, s);
      if (e != cudaSuccess) return e;
    }
    return tc_bf16_tma_gemm(c->ATb8, c->ld8V, c->Fb8, c->ld8V, c->R, c->Kp, c->D, c->Kp, c->V, c->d_status, s,
                            c->ATb8lo, c->Fb8lo);
  }
  if (c->bf16) return tc_gemm_run(a, TC_BF16, c->A_bf16, c->Kp > 128 ? 128 : 0, c->d_status, s);
  c->launch_count += c->splitR > 1;
  return gemm_run_split(a, c->ppart, c->splitR, s);
}

cudaError_t enq_product_P(nmf_ctx* c, bool operand_ready = false) {   // P = A H^T  (V x Kp)
  if (c->fmt == NMF_CSR_F32_I32) {
    c->launch_count += 1;
    return spmm_run(c->planA, c->ci, c->va, c->Ht, c->P, c->Kp, c->stream);
  }
  GemmArgs a;
  a.M = c->V; a.N = c->Kp; a.Kin = c->D;
  a.A = c->dense; a.lda = c->lda; a.transA = 0;
  a.B = c->Ht; a.ldb = c->Kp;
  a.C = c->P; a.ldc = c->Kp;
  c->launch_count += 1;
  if (c->bf16 && c->tma) {
    // P (V x Kp) = A (V x D) * (H)^T with H = (H^T)^T (Kp x D) in BF16.
    if (!operand_ready) {
      cudaError_t e = bf16_operand(c, false, c->stream);
      if (e != cudaSuccess) return e;
    }
    return tc_bf16_tma_gemm(c->Ab8, c->ld8D, c->Fb8, c->ld8D, c->P, c->Kp, c->V, c->Kp, c->D, c->d_status,
                            c->stream, c->Ab8lo, c->Fb8lo);
  }
  if (c->bf16) return tc_gemm_run(a, TC_BF16, c->A_bf16, c->Kp > 128 ? 128 : 0, c->d_status, c->stream);
  c->launch_count += c->splitP > 1;
  return gemm_run_split(a, c->ppart, c->splitP, c->stream);
}

cudaError_t enq_gram(nmf_ctx* c, const GramWork& g, const float* X, float* out, cudaStream_t s = nullptr,
                     bool operand_ready = false) {
  if (!s) s = c->stream;
  if (c->bf16 && c->tma && c->gpart) {
    // Split-K partial Grams on the tensor cores from the BF16 transposed
    // factor, then a fixed-order FP64 sum.
    const bool w = X == c->W;
    cudaError_t e;
    if (!operand_ready && (e = bf16_operand(c, w, s)) != cudaSuccess) return e;
    const int N = w ? c->V : c->D;
    const int splits = tma_gram_splits(c->Kp, N);
    c->launch_count += 2;
    if ((e = tc_bf16_tma_gram_partials(c->Fb8, w ? c->ld8V : c->ld8D, c->Kp, N, c->gpart, splits, c->d_status, s,
                                       c->Fb8lo)) !=
        cudaSuccess)
      return e;
    return gram_reduce(c->gpart, splits, c->Kp, c->K, out, s);
  }
  c->launch_count += 2;
  if (c->use_tc || c->bf16) return gram_run_tc(g, X, out, c->K, c->d_status, s, c->bf16);
  return gram_run(g, X, out, c->K, s);
}

// S = W^T W right after a W update enqueued with with_s: where the update's
// workers formed the chunk partials the Gram kernel only checks their count
// and the partials are reduced; otherwise the Gram as usual.
cudaError_t enq_gram_after_w(nmf_ctx* c, cudaStream_t s, bool shared_op) {
  if (!c->ws_gram) return enq_gram(c, c->gramW, c->W, c->S, s, shared_op);
  c->launch_count += 2;
  return gram_run(c->gramW, c->W, c->S, c->K, s ? s : c->stream, c->d_sync + w_sync_sdone_offset(c->K), c->ws_need);
}

// Regrouped update of one tall factor X (N x Kp) with Gram G and data term B.
//  H: rows are independent; one kernel runs every tile (base, chain, write).
//  W: per tile of 16 columns, a full-grid kernel forms the tile's base from the
//     current rows (new columns left of the tile, old ones right of it), then
//     the cluster kernel finishes the tile's columns with their norms.
cudaError_t enq_update(nmf_ctx* c, float* X, const float* G, const float* B, int N, bool is_w, bool pre0 = false,
                       bool with_s = false, cudaEvent_t after_chain = nullptr) {
  const int K = c->K, Kp = c->Kp;
  if (!is_w) {
    c->launch_count += 1;
    if (c->tc_updates) return h_update_tc_run(X, B, G, N, K, Kp, c->eps, c->d_status, c->stream);
    return h_update_run(X, B, G, N, K, Kp, c->eps, c->d_status, c->stream, nullptr, c->h_pack_rows);
  }
  if (c->w_persistent) {
    c->launch_count += 1;
    WPersistConfig wc = c->wp;
    wc.workers_after_chain = c->w_workers_after_chain;
    return w_persistent_run(X, B, G, c->Yc, N, K, Kp, c->eps, c->d_sync, c->d_status, wc, c->stream,
                            pre0 ? w_chain_order(c->Yc, N, c->wp).comp : nullptr, c->wait_ns, c->extra_arrivals,
                            with_s && c->ws_gram ? c->gramW.d_part : nullptr, after_chain);
  }
  // W: tile tau's base without tile tau-1 ("main") runs on the side stream
  // while the chain of tile tau-1 runs; the chain of tile tau adds tile
  // tau-1 itself.  Events: fork, base_done[tau], chain_done[tau].
  const int T = c->T;                                   // tile width of this path (<= 16)
  const int nt = (K + T - 1) / T;
  cudaEvent_t* ev = c->ev.data();
  cudaEvent_t fork = ev[0];
  cudaEvent_t* base_done = ev + 1;
  cudaEvent_t* chain_done = ev + 1 + nt;
  cudaError_t e;
  if ((e = cudaEventRecord(fork, c->stream)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c->side, fork, 0)) != cudaSuccess) return e;
  // An event wait orders against the event's latest record *in enqueue
  // order*, so every base is enqueued after the chain it depends on.
  auto base = [&](int tau) -> cudaError_t {
    const int lo = tau * T;
    const int new_end = tau >= 1 ? lo - T : 0;           // new columns [0, lo - T)
    cudaError_t err;
    if (tau >= 2 && (err = cudaStreamWaitEvent(c->side, chain_done[tau - 2], 0)) != cudaSuccess) return err;
    if ((err = w_prep_run(X, B, G, c->Y, N, K, Kp, lo, new_end, c->d_status, c->side, T)) != cudaSuccess)
      return err;
    c->launch_count += 1;
    return cudaEventRecord(base_done[tau], c->side);
  };
  if ((e = base(0)) != cudaSuccess) return e;
  if (nt > 1 && (e = base(1)) != cudaSuccess) return e;
  for (int tau = 0; tau < nt; ++tau) {
    const int lo = tau * T, hi = std::min(K, lo + T);
    if ((e = cudaStreamWaitEvent(c->stream, base_done[tau], 0)) != cudaSuccess) return e;
    e = chain_run(c->Y, X, G, N, Kp, lo, hi, tau >= 1 ? lo - T : -1, c->eps, true, c->chainW, c->d_status,
                  c->stream);
    c->launch_count += 1;
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(chain_done[tau], c->stream)) != cudaSuccess) return e;
    // Base of tile tau + 2 (needs chains <= tau) overlaps the chain of tau + 1.
    if (tau + 2 < nt && (e = base(tau + 2)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t enq_objective(nmf_ctx* c) {
  c->launch_count += 3;
  return objective_run(c->W, c->P, c->V, c->Kp, c->S, c->Q, c->normA2, c->obj_partial,
                       c->n_obj_partial, c->hist, c->d_counter, kHistCap, c->stream);
}

// One iteration.  On entry S = W^T W and R = A^T W for the current W (the
// first two products of Alg. 1); on exit the same holds for the new W.  R is therefore formed at
// the end of the previous iteration, right after the W update, where it runs
// beside S; likewise Q beside P.  Each pair is independent (same inputs,
// disjoint outputs and work buffers), so the graph has two branches there:
//   H update -> { P | Q } -> W update -> { S -> objective | R | <W, P> }
// (the objective's <W, P> part needs only the new W and P, so it runs on a
// third branch and the objective's last step only adds <S, Q>).
// Host copies folded into one iteration (nmf_iterate_host): the new H is
// copied out on side3 while P, Q and the W update run, the new W once the W
// update is done (beside S and the objective), and the objective after it;
// R of the new W, which the next iteration would need, is not formed (the
// caller brings a new W).
struct IoHooks {
  float* H_out = nullptr;      // host, K x D
  float* W_out = nullptr;      // host, V x K
  double* obj_host = nullptr;  // pinned host scalar
};

cudaError_t enq_iteration(nmf_ctx* c, const IoHooks* io = nullptr) {
  cudaError_t e;
  cudaStream_t m = c->stream, b = c->side;
  const bool shared_op = c->bf16 && c->tma;      // one BF16 factor operand for both branches
  if ((e = enq_update(c, c->Ht, c->S, c->R, c->D, false)) != cudaSuccess) return e;
  if (io && io->H_out) {
    if ((e = cudaEventRecord(c->evio[0], m)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->side3, c->evio[0], 0)) != cudaSuccess) return e;
    c->launch_count += 1;
    if ((e = transpose_f32(c->Ht, c->D, c->K, c->Kp, c->stage, c->D, c->side3)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(io->H_out, c->stage, sizeof(float) * (size_t)c->K * c->D, cudaMemcpyDefault,
                             c->side3)) != cudaSuccess)
      return e;
  }
  if (shared_op && (e = bf16_operand(c, false, m)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(c->evx[0], m)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(b, c->evx[0], 0)) != cudaSuccess) return e;
  if ((e = enq_gram(c, c->gramH, c->Ht, c->Q, b, shared_op)) != cudaSuccess) return e;
  // Persistent W update: tile 0's base less P (it needs Q and the old W
  // only) on this branch, while P is still running.
  const bool pre0 = c->w_persistent;
  if (pre0) {
    c->launch_count += 1;
    const ChainOrder co = w_chain_order(c->Yc, c->V, c->wp);
    if ((e = w_prep_run(c->W, nullptr, c->Q, nullptr, c->V, c->K, c->Kp, 0, 0, c->d_status, b, kRowTile, nullptr,
                        &co)) != cudaSuccess)
      return e;
  }
  if ((e = cudaEventRecord(c->evx[1], b)) != cudaSuccess) return e;
  if ((e = enq_product_P(c, shared_op)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(m, c->evx[1], 0)) != cudaSuccess) return e;
  // The steps that read only the new W (R, <W, P>, the copy-out) start when
  // the W update's chain grid is done, beside the workers' last block
  // columns of S (the grid that follows it on this stream).
  const bool early = c->w_persistent && !shared_op;
  if ((e = enq_update(c, c->W, c->Q, c->P, c->V, true, pre0, true, early ? c->evx[5] : nullptr)) != cudaSuccess)
    return e;
  if (shared_op && (e = bf16_operand(c, true, m)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(c->evx[2], m)) != cudaSuccess) return e;
  const cudaEvent_t w_ready = early ? c->evx[5] : c->evx[2];
  if (!io) {
    if ((e = cudaStreamWaitEvent(b, w_ready, 0)) != cudaSuccess) return e;
    if ((e = enq_product_R(c, b, shared_op)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->evx[3], b)) != cudaSuccess) return e;
  } else if (io->W_out) {
    if ((e = cudaStreamWaitEvent(c->side3, w_ready, 0)) != cudaSuccess) return e;
    if ((e = cudaMemcpy2DAsync(io->W_out, sizeof(float) * c->K, c->W, sizeof(float) * c->Kp, sizeof(float) * c->K,
                               c->V, cudaMemcpyDefault, c->side3)) != cudaSuccess)
      return e;
  }
  if ((e = cudaStreamWaitEvent(c->side2, w_ready, 0)) != cudaSuccess) return e;
  c->launch_count += 3;
  if ((e = objective_wp(c->W, c->P, c->V, c->Kp, c->obj_partial, c->n_obj_partial, c->side2)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(c->evx[4], c->side2)) != cudaSuccess) return e;
  if ((e = enq_gram_after_w(c, nullptr, shared_op)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(m, c->evx[4], 0)) != cudaSuccess) return e;
  if ((e = objective_finish(c->Kp, c->S, c->Q, c->normA2, c->obj_partial, c->n_obj_partial, c->hist, c->d_counter,
                            kHistCap, m, io ? c->d_obj_last : nullptr)) != cudaSuccess)
    return e;
  if (!io) return cudaStreamWaitEvent(m, c->evx[3], 0);
  if (io->obj_host &&
      (e = cudaMemcpyAsync(io->obj_host, c->d_obj_last, sizeof(double), cudaMemcpyDeviceToHost, m)) != cudaSuccess)
    return e;
  if ((e = cudaEventRecord(c->evio[1], c->side3)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(m, c->evio[1], 0);
}

// Establish the iteration's entry state (S and R of the current W).
cudaError_t ensure_entry(nmf_ctx* c) {
  cudaError_t e;
  if (!c->s_valid) {
    if ((e = enq_gram(c, c->gramW, c->W, c->S)) != cudaSuccess) return e;
    c->s_valid = true;
  }
  if (!c->r_valid) {
    if ((e = enq_product_R(c)) != cudaSuccess) return e;
    c->r_valid = true;
  }
  return cudaSuccess;
}

nmf_status read_status(nmf_ctx* c) {
  int st = 0;
  CK(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    CK(cudaMemset(c->d_status, 0, sizeof(int)));
    if (st & ST_TIMEOUT) return NMF_ETIMEOUT;
    if (st & ST_NUMERIC) return NMF_ENUMERIC;
  }
  return NMF_OK;
}

void destroy_graph(nmf_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  if (c->graph_alg1_exec) cudaGraphExecDestroy(c->graph_alg1_exec);
  if (c->graph_alg1) cudaGraphDestroy(c->graph_alg1);
  c->graph_alg1_exec = nullptr;
  c->graph_alg1 = nullptr;
  if (c->graph_mu_exec) cudaGraphExecDestroy(c->graph_mu_exec);
  if (c->graph_mu) cudaGraphDestroy(c->graph_mu);
  c->graph_mu_exec = nullptr;
  c->graph_mu = nullptr;
  if (c->graph_io_exec) cudaGraphExecDestroy(c->graph_io_exec);
  if (c->graph_io) cudaGraphDestroy(c->graph_io);
  c->graph_io_exec = nullptr;
  c->graph_io = nullptr;
}

nmf_status validate_and_copy_csr(const nmf_problem* p, std::vector<int>& rp, std::vector<int>& ci,
                                 std::vector<float>& va, double* normA2) {
  if (!p->row_ptr || (p->nnz > 0 && (!p->col_idx || !p->val)) || p->nnz < 0) return NMF_EINVAL;
  if (p->nnz > 0x7fffffffLL) return NMF_EUNSUPPORTED;
  rp.resize((size_t)p->V + 1);
  ci.resize((size_t)p->nnz);
  va.resize((size_t)p->nnz);
  CK(cudaMemcpy(rp.data(), p->row_ptr, sizeof(int) * rp.size(), cudaMemcpyDefault));
  if (p->nnz > 0) {
    CK(cudaMemcpy(ci.data(), p->col_idx, sizeof(int) * ci.size(), cudaMemcpyDefault));
    CK(cudaMemcpy(va.data(), p->val, sizeof(float) * va.size(), cudaMemcpyDefault));
  }
  if (rp[0] != 0 || rp[p->V] != p->nnz) return NMF_EINVAL;
  for (int r = 0; r < p->V; ++r)
    if (rp[r + 1] < rp[r]) return NMF_EINVAL;
  double s = 0.0;
  for (int64_t e = 0; e < p->nnz; ++e) {
    if (ci[e] < 0 || ci[e] >= p->D) return NMF_EINVAL;
    const float v = va[e];
    if (!(v >= 0.f) || !std::isfinite(v)) return NMF_EINVAL;
    s += (double)v * (double)v;
  }
  *normA2 = s;
  return NMF_OK;
}

nmf_status init_impl(const nmf_problem* p, nmf_ctx* c) {
  c->V = p->V;
  c->D = p->D;
  c->K = p->K;
  c->Kp = (p->K + 3) & ~3;
  c->fmt = p->fmt;
  c->prec = p->prec;
  c->eps = p->eps == 0.f ? 1e-16f : p->eps;
  const int V = c->V, D = c->D, Kp = c->Kp;
  if (p->stream) {
    c->stream = static_cast<cudaStream_t>(p->stream);
  } else {
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  // Tile width T of the regrouped updates: 16 columns (the register tile of
  // the column chain).  With the per-tile W launches (NMF_FLAG_MULTI_LAUNCH_W)
  // a requested tile_T of 1..16 sets the W update's tile width (the tile-size
  // study; the H update keeps 16); otherwise a request is taken as one for
  // the library choice.
  const int T = (p->flags & NMF_FLAG_MULTI_LAUNCH_W) && p->tile_T >= 1 && p->tile_T <= kRowTile ? p->tile_T
                                                                                              : kRowTile;
  if (!chain_config_for(V, true, T, &c->chainW)) return NMF_EUNSUPPORTED;
  if (!chain_config_for(D, false, T, &c->chainH)) return NMF_EUNSUPPORTED;
  c->T = T;

  CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&c->side3, cudaStreamNonBlocking));
  {
    const int nt = (c->K + T - 1) / T;
    c->ev.assign(1 + 2 * nt, nullptr);
    for (auto& e : c->ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : c->evx) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : c->evio) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  CK(dalloc(&c->d_obj_last, 1));
  CK(cudaHostAlloc(reinterpret_cast<void**>(&c->h_obj), sizeof(double), cudaHostAllocDefault));
  CK(cudaHostAlloc(reinterpret_cast<void**>(&c->h_status), sizeof(int), cudaHostAllocDefault));
  CK(dalloc(&c->d_status, 1));
  CK(cudaMemset(c->d_status, 0, sizeof(int)));
  CK(dalloc(&c->d_sync, w_sync_ints(c->K)));
  CK(dalloc(&c->d_counter, 1));
  CK(cudaMemset(c->d_counter, 0, sizeof(unsigned)));
  CK(dalloc(&c->hist, kHistCap));
  CK(dalloc(&c->obj_partial, 2 * c->n_obj_partial));

  if (c->fmt == NMF_CSR_F32_I32) {
    std::vector<int> rp, ci;
    std::vector<float> va;
    nmf_status st = validate_and_copy_csr(p, rp, ci, va, &c->normA2);
    if (st != NMF_OK) return st;
    c->rp = p->row_ptr;
    c->ci = p->col_idx;
    c->va = p->val;
    c->nnz = p->nnz;
    // CSR of A^T (documents as rows), built by a stable counting sort so
    // that word indices stay ascending inside every document row.
    std::vector<int> rpT((size_t)D + 1, 0), ciT((size_t)p->nnz);
    std::vector<float> vaT((size_t)p->nnz);
    for (int64_t e = 0; e < p->nnz; ++e) rpT[(size_t)ci[e] + 1]++;
    for (int d = 0; d < D; ++d) rpT[d + 1] += rpT[d];
    std::vector<int> fill(rpT.begin(), rpT.end() - 1);
    for (int r = 0; r < V; ++r)
      for (int e = rp[r]; e < rp[r + 1]; ++e) {
        const int pos = fill[ci[e]]++;
        ciT[pos] = r;
        vaT[pos] = va[e];
      }
    CK(dalloc(&c->rpT, rpT.size()));
    CK(dalloc(&c->ciT, ciT.size()));
    CK(dalloc(&c->vaT, vaT.size()));
    CK(cudaMemcpy(c->rpT, rpT.data(), sizeof(int) * rpT.size(), cudaMemcpyHostToDevice));
    if (p->nnz > 0) {
      CK(cudaMemcpy(c->ciT, ciT.data(), sizeof(int) * ciT.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->vaT, vaT.data(), sizeof(float) * vaT.size(), cudaMemcpyHostToDevice));
    }
    CK(spmm_plan_build(c->planA, rp, V, D, Kp, c->segA));
    CK(spmm_plan_build(c->planAt, rpT, D, V, Kp, c->segAt));
    c->h_rp = std::move(rp);
    c->h_rpT = std::move(rpT);
  } else if (c->fmt == NMF_DENSE_F32) {
    if (!p->dense || p->ld < p->D) return NMF_EINVAL;
    if (!is_device_ptr(p->dense)) return NMF_EINVAL;
    c->dense = p->dense;
    c->lda = p->ld;
    // Small products: split K so that every SM has work (R is D x Kp over V,
    // P is V x Kp over D); the two never run at the same time.
    c->splitR = splitk_chunks(D, Kp, V);
    c->splitP = splitk_chunks(V, Kp, D);
    if (c->splitR > 1 || c->splitP > 1)
      CK(dalloc(&c->ppart, std::max((size_t)c->splitR * D, (size_t)c->splitP * V) * Kp));
    double* d_part = nullptr;
    int* d_bad = nullptr;
    CK(dalloc(&d_part, kSumsqBlocks));
    CK(dalloc(&d_bad, 1));
    CK(cudaMemset(d_bad, 0, sizeof(int)));
    CK(sumsq_dense_f64(p->dense, V, D, p->ld, d_part, d_bad, c->stream));
    std::vector<double> part(kSumsqBlocks);
    int bad = 0;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(part.data(), d_part, sizeof(double) * kSumsqBlocks, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(d_part);
    cudaFree(d_bad);
    if (bad) return NMF_EINVAL;
    double s = 0.0;
    for (double v : part) s += v;
    c->normA2 = s;
  } else {
    return NMF_EINVAL;
  }
  if (!(c->normA2 > 0.0)) return NMF_EINVAL;

  const size_t nV = (size_t)V * Kp, nD = (size_t)D * Kp, nK = (size_t)Kp * Kp;
  const size_t nMax = (size_t)std::max(V, D) * Kp;
  CK(dalloc(&c->W, nV));
  CK(dalloc(&c->P, nV));
  CK(dalloc(&c->Ht, nD));
  CK(dalloc(&c->R, nD));
  CK(dalloc(&c->S, nK));
  CK(dalloc(&c->Q, nK));
  CK(dalloc(&c->Y, nMax));
  CK(dalloc(&c->stage, nMax));
  CK(dalloc(&c->alg1_part, (size_t)alg1_parts(V)));
  CK(cudaMemsetAsync(c->P, 0, sizeof(float) * nV, c->stream));
  CK(cudaMemsetAsync(c->R, 0, sizeof(float) * nD, c->stream));
  CK(cudaMemsetAsync(c->Y, 0, sizeof(float) * nMax, c->stream));
  c->use_tc = (p->flags & NMF_FLAG_TC_GRAMS) != 0;
  c->tc_updates = (p->flags & NMF_FLAG_TC_UPDATES) && h_update_tc_supported(Kp) && tma_available();
  c->bf16 = c->prec == NMF_PREC_BF16;
  if (c->bf16) {
    // BF16 copy of A for the tensor-core products; FP32 Grams and buffers for
    // the objective against the FP32 A (nmf_error).
    c->tma = tma_available() && !(p->flags & NMF_FLAG_NO_TMA);
    if (!c->tma) {
      CK(cudaMalloc(&c->A_bf16, sizeof(uint16_t) * (size_t)V * c->lda));
      CK(convert_bf16(c->dense, V, D, c->lda, c->A_bf16, c->lda, c->stream));
    } else {
      c->ld8V = (V + 7) / 8 * 8;
      c->ld8D = (D + 7) / 8 * 8;
      CK(cudaMalloc(&c->Ab8, sizeof(uint16_t) * (size_t)V * c->ld8D));
      CK(cudaMalloc(&c->ATb8, sizeof(uint16_t) * (size_t)D * c->ld8V));
      if (!(p->flags & NMF_FLAG_BF16_SINGLE_A)) {
        CK(cudaMalloc(&c->Ab8lo, sizeof(uint16_t) * (size_t)V * c->ld8D));
        CK(cudaMalloc(&c->ATb8lo, sizeof(uint16_t) * (size_t)D * c->ld8V));
      }
      CK(cudaMalloc(&c->Fb8, sizeof(uint16_t) * (size_t)Kp * std::max(c->ld8V, c->ld8D)));
      if (c->Ab8lo && !(p->flags & NMF_FLAG_BF16_SINGLE_FACTORS))
        CK(cudaMalloc(&c->Fb8lo, sizeof(uint16_t) * (size_t)Kp * std::max(c->ld8V, c->ld8D)));
      c->gsplits = std::max(tma_gram_splits(Kp, V), tma_gram_splits(Kp, D));
      CK(cudaMalloc(&c->gpart, sizeof(float) * (size_t)c->gsplits * Kp * Kp));
      // A (V x D) -> BF16 with row stride ld8D, and A^T (D x V) with ld8V.
      CK(convert_bf16(c->dense, V, D, c->lda, c->Ab8, c->ld8D, c->stream, c->Ab8lo));
      CK(transpose_to_bf16(c->dense, V, D, c->lda, c->ATb8, c->ld8V, c->stream, c->ATb8lo));
    }
  }
  if (c->fmt == NMF_DENSE_F32) CK(dalloc(&c->resid_part, (size_t)resid2_partials(V, D)));
  if (c->use_tc || c->bf16) {
    CK(gram_setup_tc(c->gramW, V, Kp));
    CK(gram_setup_tc(c->gramH, D, Kp));
  } else {
    CK(gram_setup(c->gramW, V, Kp));
    CK(gram_setup(c->gramH, D, Kp));
  }

  // Initial factors.
  const uint64_t sw = p->seed ^ 0x5757575757575757ull, sh = p->seed ^ 0x4848484848484848ull;
  if (p->W0) {
    CK(cudaMemsetAsync(c->W, 0, sizeof(float) * nV, c->stream));
    CK(cudaMemcpy2DAsync(c->W, sizeof(float) * Kp, p->W0, sizeof(float) * p->K, sizeof(float) * p->K, V,
                         cudaMemcpyDefault, c->stream));
  } else {
    CK(fill_uniform_splitmix(c->W, V, p->K, Kp, sw, c->stream));
  }
  if (p->H0) {
    CK(cudaMemcpyAsync(c->stage, p->H0, sizeof(float) * (size_t)p->K * D, cudaMemcpyDefault, c->stream));
    CK(cudaMemsetAsync(c->Ht, 0, sizeof(float) * nD, c->stream));
    CK(transpose_f32(c->stage, p->K, D, D, c->Ht, Kp, c->stream));
  } else {
    CK(fill_uniform_splitmix_t(c->Ht, D, p->K, Kp, sh, c->stream));
  }
  CK(normalize_columns(c->W, V, p->K, Kp, c->stream));
  // Whole W update in one launch wherever a 16- or 8-CTA chain cluster and at
  // least one worker cluster fit; its result does not depend on how many of
  // the clusters run at the same time, so no probe launch is needed.
  c->w_persistent = !(p->flags & NMF_FLAG_MULTI_LAUNCH_W) && w_persistent_config(V, Kp, &c->wp, c->tc_updates);
  if (c->w_persistent) {
    CK(dalloc(&c->Yc, w_chain_base_floats()));
    CK(cudaMemsetAsync(c->Yc, 0, sizeof(float) * w_chain_base_floats(), c->stream));
  }
  c->gramW0 = c->gramW;
  if (c->w_persistent && !c->wp.tc && !c->use_tc && !c->bf16 && Kp <= 256 && gram_tri_single_group(c->gramW) &&
      (size_t)c->wp.worker_rows * (Kp + 4) >= 16 * 256) {
    int nb = 0, per = 0;
    w_persistent_blocks(V, c->wp, &nb, &per);
    if (nb >= 1 && nb <= c->gramW0.n_chunks) {
      // gramW chunked by the workers' row blocks (its partial buffer holds
      // gramW0.n_chunks >= nb chunks).
      gram_rechunk(c->gramW, per, nb);
      c->ws_gram = true;
      c->ws_need = nb * ((c->K + kRowTile - 1) / kRowTile);
    }
  }
  CK(enq_gram(c, c->gramW, c->W, c->S));
  c->s_valid = true;
  CK(cudaStreamSynchronize(c->stream));
  // Count the launches of one iteration (dry count, nothing is enqueued).
  return NMF_OK;
}

void free_ctx(nmf_ctx* c) {
  if (!c) return;
  destroy_graph(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  spmm_plan_free(c->planA);
  spmm_plan_free(c->planAt);
  gram_free(c->gramW);
  gram_free(c->gramH);

  for (void* p : {(void*)c->A_bf16, c->Ab8, c->ATb8, c->Ab8lo, c->ATb8lo, c->Fb8, c->Fb8lo, (void*)c->gpart, (void*)c->ppart, (void*)c->resid_part,
                  (void*)c->d_sync, (void*)c->rpT, (void*)c->ciT, (void*)c->vaT, (void*)c->W, (void*)c->Ht, (void*)c->R,
                  (void*)c->P, (void*)c->S, (void*)c->Q, (void*)c->Y, (void*)c->stage, (void*)c->Yc, (void*)c->alg1_part,
                  (void*)c->obj_partial, (void*)c->hist, (void*)c->d_counter, (void*)c->d_status,
                  (void*)c->d_obj_last})
    if (p) cudaFree(p);
  if (c->h_obj) cudaFreeHost(c->h_obj);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->side3) {
    cudaStreamSynchronize(c->side3);
    cudaStreamDestroy(c->side3);
  }
  for (auto e : c->evio)
    if (e) cudaEventDestroy(e);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->side2) {
    cudaStreamSynchronize(c->side2);
    cudaStreamDestroy(c->side2);
  }
  for (auto e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto e : c->evx)
    if (e) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace

// ---------------------------------------------------------------------------
// Batched form: independent problems advanced together.  One CUDA graph holds
// one iteration of every member, each member's launches on its own stream
// (graph branches joined at the end), so the hardware runs the members'
// kernels side by side on the SMs one small problem leaves idle.  Members
// use the per-tile W launches: the persistent W kernel occupies every SM.
// ---------------------------------------------------------------------------
struct nmf_batch {
  std::vector<nmf_ctx*> m;
  cudaStream_t root = nullptr;
  bool own_root = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join, ready;
  std::vector<float> w_us;        // autotuner: W update time of the chosen configuration
};

namespace {

void free_batch(nmf_batch* b) {
  if (!b) return;
  if (b->root) cudaStreamSynchronize(b->root);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->join) if (e) cudaEventDestroy(e);
  for (auto e : b->ready) if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->own_root && b->root) cudaStreamDestroy(b->root);
  delete b;
}

// Drop a member's cached single-problem graph (it is re-captured on the next
// nmf_iterate with the member's current W configuration).
void drop_graph(nmf_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  if (c->graph_io_exec) cudaGraphExecDestroy(c->graph_io_exec);
  if (c->graph_io) cudaGraphDestroy(c->graph_io);
  c->graph_io_exec = nullptr;
  c->graph_io = nullptr;
}

// SpMM schedule of one product (which = 0: P = A H^T over the CSR of A,
// 1: R = A^T W over the CSR of A^T): its plan rebuilt with rows longer than
// seg non-zeros split into seg-long items (seg = kNoSplit: one item per row).
constexpr int kNoSplit = 1 << 30;
cudaError_t set_spmm_seg(nmf_ctx* c, int which, int seg) {
  SpmmPlan& plan = which == 0 ? c->planA : c->planAt;
  spmm_plan_free(plan);
  cudaError_t e = which == 0 ? spmm_plan_build(plan, c->h_rp, c->V, c->D, c->Kp, seg)
                             : spmm_plan_build(plan, c->h_rpT, c->D, c->V, c->Kp, seg);
  if (e != cudaSuccess) return e;
  (which == 0 ? c->segA : c->segAt) = seg;
  return cudaSuccess;
}

// Times each product with seg in {128, 256, 512, 1024, no split} (CUDA
// events on the context's stream, the current factors; one warm-up and
// three timed runs each) and keeps the fastest.  The products' outputs are
// overwritten (P with A H^T of the current H, R with A^T W of the current
// W, the last one with the chosen plan).
cudaError_t tune_spmm_segs(nmf_ctx* c) {
  if (c->fmt != NMF_CSR_F32_I32) return cudaSuccess;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  const int segs[] = {128, 256, 512, 1024, kNoSplit};
  for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
    const int* ci = which == 0 ? c->ci : c->ciT;
    const float* va = which == 0 ? c->va : c->vaT;
    const float* X = which == 0 ? c->Ht : c->W;
    float* Y = which == 0 ? c->P : c->R;
    int best_seg = which == 0 ? c->segA : c->segAt;
    float best = INFINITY;
    for (int seg : segs) {
      if ((e = set_spmm_seg(c, which, seg)) != cudaSuccess) break;
      const SpmmPlan& plan = which == 0 ? c->planA : c->planAt;
      for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(t0, c->stream);
        if (e == cudaSuccess) e = spmm_run(plan, ci, va, X, Y, c->Kp, c->stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(t1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        best_seg = seg;
      }
    }
    if (e == cudaSuccess) e = set_spmm_seg(c, which, best_seg);
  }
  if (e == cudaSuccess) e = enq_product_R(c);          // R of the current W with the chosen plan
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  return e;
}

// Autotuner for a batch member (Sec. 1's repeated factorisation: many small
// problems of uneven shape, each with its own best schedule).  Three choices
// are timed per member with CUDA events, each from the same start:
//  * the SpMM schedule of each product (CSR SpMM of A for P, of A^T for R):
//    rows longer than `seg` non-zeros are split into seg-long items whose
//    partial rows the last item sums; seg in {128, 256, 512, 1024} or no
//    split at all (one item per row); the fastest of three runs each wins;
//  * the W update's column-tile width T in {8, 12, 16} (Alg. 2's T; each tile
//    costs a base launch and a chain launch, each column a cluster-wide norm)
//    and the chain's cluster size (4, 8 or 16 CTAs: a wider cluster finishes
//    the chain sooner but holds more SMs the other members could use): the
//    pair with the least chain SM-time (CTAs x microseconds of three
//    updates) wins.
// W is restored afterwards and R is recomputed for the current W, so tuning
// does not advance the factorisation.
cudaError_t autotune_member(nmf_ctx* c, float* w_us_out) {
  const size_t bytes = sizeof(float) * (size_t)c->V * c->Kp;
  float* saved = nullptr;
  cudaError_t e = cudaMalloc(&saved, bytes);
  if (e != cudaSuccess) return e;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  auto fail = [&](cudaError_t err) {
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(saved);
    return err;
  };
  if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) return fail(e);
  auto elapsed_us = [&](int reps, float* us) -> cudaError_t {
    cudaError_t err;
    if ((err = cudaEventRecord(t1, c->stream)) != cudaSuccess) return err;
    if ((err = cudaEventSynchronize(t1)) != cudaSuccess) return err;
    float ms = 0.f;
    if ((err = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess) return err;
    *us = ms * 1000.f / (float)reps;
    return cudaSuccess;
  };
  // SpMM schedules (sparse A only).
  if ((e = tune_spmm_segs(c)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(saved, c->W, bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) return fail(e);
  // P and Q of the current H: the W update's inputs.
  if ((e = enq_product_P(c)) != cudaSuccess) return fail(e);
  if ((e = enq_gram(c, c->gramH, c->Ht, c->Q)) != cudaSuccess) return fail(e);
  ChainConfig best = c->chainW;
  int best_T = c->T;
  float best_cost = INFINITY, best_us = 0.f;
  for (int T : {16, 12, 8}) {
    // Events of the per-tile launches: 1 + 2 * ceil(K / T).
    const size_t need = 1 + 2 * (size_t)((c->K + T - 1) / T);
    while (c->ev.size() < need) {
      cudaEvent_t ev = nullptr;
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
      c->ev.push_back(ev);
    }
    for (int cl : {16, 8, 4}) {
      ChainConfig cfg;
      if (!chain_config_cluster(c->V, T, cl, &cfg)) continue;
      c->chainW = cfg;
      c->T = T;
      // warm-up, then three timed updates
      for (int rep = 0; rep < 4; ++rep) {
        if ((e = cudaMemcpyAsync(c->W, saved, bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
          return fail(e);
        if (rep == 1 && (e = cudaEventRecord(t0, c->stream)) != cudaSuccess) return fail(e);
        if ((e = enq_update(c, c->W, c->Q, c->P, c->V, true)) != cudaSuccess) return fail(e);
      }
      float us = 0.f;      // includes the three restoring copies (the same for every choice)
      if ((e = elapsed_us(3, &us)) != cudaSuccess) return fail(e);
      const float cost = us * (float)cl;
      if (cost < best_cost) {
        best_cost = cost;
        best = cfg;
        best_T = T;
        best_us = us;
      }
    }
  }
  c->chainW = best;
  c->T = best_T;
  *w_us_out = best_us;
  if ((e = cudaMemcpyAsync(c->W, saved, bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) return fail(e);
  // R = A^T W of the restored W (the iteration's entry state).
  if ((e = enq_product_R(c)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return fail(e);
  return fail(cudaSuccess);
}

}  // namespace

extern "C" {

nmf_status nmf_batch_create(nmf_ctx* const* ctxs, int32_t n, int32_t autotune, void* stream, nmf_batch** out) {
  if (!ctxs || n < 1 || !out) return NMF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return NMF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream) return NMF_EINVAL;
  }
  nmf_batch* b = new (std::nothrow) nmf_batch;
  if (!b) return NMF_ENOMEM;
  b->m.assign(ctxs, ctxs + n);
  b->w_us.assign(n, 0.f);
  cudaError_t e = cudaSuccess;
  auto bail = [&](cudaError_t err) {
    cudaGetLastError();
    free_batch(b);
    return from_cuda(err);
  };
  if (stream) {
    b->root = static_cast<cudaStream_t>(stream);
    for (auto* c : b->m)
      if (c->stream == b->root) {
        free_batch(b);
        return NMF_EINVAL;
      }
  } else {
    if ((e = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    b->own_root = true;
  }
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return bail(e);
  if ((e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess) return bail(e);
  b->join.assign(n, nullptr);
  b->ready.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    if ((e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming)) != cudaSuccess) return bail(e);
    if ((e = cudaEventCreateWithFlags(&b->ready[i], cudaEventDisableTiming)) != cudaSuccess) return bail(e);
  }
  for (int i = 0; i < n; ++i) {
    nmf_ctx* c = b->m[i];
    c->w_persistent = false;
    c->h_pack_rows = true;        // the members share the SMs: fewer, fuller CTAs (same arithmetic)
    if (c->ws_gram) {
      // The per-tile W update forms no Gram partials; S is formed again with
      // the Gram's own chunking, so that a member computes exactly what a
      // context made for the per-tile form does.
      c->ws_gram = false;
      c->gramW = c->gramW0;
      c->s_valid = false;
    }
    drop_graph(c);
    if ((e = ensure_entry(c)) != cudaSuccess) return bail(e);
    if (autotune) {
      if ((e = autotune_member(c, &b->w_us[i])) != cudaSuccess) return bail(e);
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e);
  }
  // Capture one iteration of every member as branches of one graph.
  if ((e = cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return bail(e);
  cudaError_t ce = cudaEventRecord(b->fork, b->root);
  for (int i = 0; i < n && ce == cudaSuccess; ++i) {
    nmf_ctx* c = b->m[i];
    if ((ce = cudaStreamWaitEvent(c->stream, b->fork, 0)) != cudaSuccess) break;
    c->launch_count = 0;
    if ((ce = enq_iteration(c)) != cudaSuccess) break;
    c->launches_per_iter = c->launch_count;
    if ((ce = cudaEventRecord(b->join[i], c->stream)) != cudaSuccess) break;
    ce = cudaStreamWaitEvent(b->root, b->join[i], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->root, &g);
  if (ce != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bail(ce != cudaSuccess ? ce : e);
  }
  b->graph = g;
  if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) return bail(e);
  *out = b;
  return NMF_OK;
}

nmf_status nmf_batch_iterate(nmf_batch* b, int32_t n_iters) {
  if (!b || n_iters < 0) return NMF_EINVAL;
  if (n_iters == 0) return NMF_OK;
  const int n = (int)b->m.size();
  // Entry state of every member (S, R of its current W), then order after
  // whatever the members' own streams hold (factor uploads, ...).
  for (int i = 0; i < n; ++i) CK(ensure_entry(b->m[i]));
  for (int i = 0; i < n; ++i) {
    CK(cudaEventRecord(b->ready[i], b->m[i]->stream));
    CK(cudaStreamWaitEvent(b->root, b->ready[i], 0));
  }
  for (int it = 0; it < n_iters; ++it) CK(cudaGraphLaunch(b->exec, b->root));
  CK(cudaEventRecord(b->done, b->root));
  for (auto* c : b->m) {
    CK(cudaStreamWaitEvent(c->stream, b->done, 0));
    c->iters_run += n_iters;
  }
  return NMF_OK;
}

nmf_status nmf_batch_query(nmf_batch* b, int32_t i, int32_t* chain_ctas, float* w_update_us) {
  if (!b || i < 0 || i >= (int)b->m.size()) return NMF_EINVAL;
  if (chain_ctas) *chain_ctas = b->m[i]->chainW.cluster;
  if (w_update_us) *w_update_us = b->w_us[i];
  return NMF_OK;
}

nmf_status nmf_batch_query_schedule(nmf_batch* b, int32_t i, int32_t* tile_T, int32_t* spmm_seg_P,
                                    int32_t* spmm_seg_R) {
  if (!b || i < 0 || i >= (int)b->m.size()) return NMF_EINVAL;
  const nmf_ctx* c = b->m[i];
  const bool sparse = c->fmt == NMF_CSR_F32_I32;
  if (tile_T) *tile_T = c->T;
  if (spmm_seg_P) *spmm_seg_P = sparse ? c->segA : 0;
  if (spmm_seg_R) *spmm_seg_R = sparse ? c->segAt : 0;
  return NMF_OK;
}

void nmf_batch_destroy(nmf_batch* b) { free_batch(b); }

nmf_status nmf_batch_submit(const nmf_problem* ps, int32_t n, int32_t n_iters, nmf_ctx** outs) {
  if (!ps || n < 1 || n_iters < 0 || !outs) return NMF_EINVAL;
  for (int i = 0; i < n; ++i) outs[i] = nullptr;
  auto undo = [&](nmf_status st) {
    for (int i = 0; i < n; ++i) {
      nmf_destroy(outs[i]);
      outs[i] = nullptr;
    }
    return st;
  };
  for (int i = 0; i < n; ++i) {
    const nmf_status st = nmf_init(&ps[i], &outs[i]);
    if (st != NMF_OK) return undo(st);
  }
  nmf_batch* b = nullptr;
  nmf_status st = nmf_batch_create(outs, n, 1, nullptr, &b);
  if (st != NMF_OK) return undo(st);
  st = nmf_batch_iterate(b, n_iters);
  nmf_batch_destroy(b);       // waits for the batch's launches
  return st == NMF_OK ? NMF_OK : undo(st);
}

}  // extern "C"

extern "C" {

const char* nmf_status_str(int32_t s) {
  switch (s) {
    case NMF_OK: return "ok";
    case NMF_EINVAL: return "invalid argument";
    case NMF_ENOMEM: return "out of device memory";
    case NMF_ECUDA: return "CUDA error";
    case NMF_ETIMEOUT: return "device wait timed out";
    case NMF_ENUMERIC: return "zero or non-finite column norm";
    case NMF_EBUSY: return "context busy";
    case NMF_EUNSUPPORTED: return "unsupported by this build";
    default: return "unknown status";
  }
}

nmf_status nmf_init(const nmf_problem* p, nmf_ctx** out) {
  if (!p || !out) return NMF_EINVAL;
  *out = nullptr;
  if (p->V <= 0 || p->D <= 0 || p->K <= 0 || p->K > std::min(p->V, p->D)) return NMF_EINVAL;
  if (p->K > kMaxK) return NMF_EUNSUPPORTED;
  if (!(p->eps >= 0.f) || !std::isfinite(p->eps)) return NMF_EINVAL;
  if (p->tile_T < 0) return NMF_EINVAL;
  if (p->prec != NMF_PREC_FP32 && p->prec != NMF_PREC_BF16) return NMF_EINVAL;
  if (p->prec == NMF_PREC_BF16 && p->fmt != NMF_DENSE_F32) return NMF_EUNSUPPORTED;
  nmf_ctx* c = new (std::nothrow) nmf_ctx();
  if (!c) return NMF_ENOMEM;
  nmf_status st = init_impl(p, c);
  if (st != NMF_OK) {
    cudaGetLastError();
    free_ctx(c);
    return st;
  }
  *out = c;
  return NMF_OK;
}

nmf_status nmf_iterate(nmf_ctx* c, int32_t n_iters) {
  if (!c || n_iters < 0) return NMF_EINVAL;
  if (n_iters == 0) return NMF_OK;
  c->launch_count = 0;
  CK(ensure_entry(c));
  if (!c->graph_exec) {
    c->launch_count = 0;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enq_iteration(c);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return from_cuda(e != cudaSuccess ? e : e2);
    }
    c->graph = g;
    c->launches_per_iter = c->launch_count;
    CK(cudaGraphInstantiate(&c->graph_exec, g, 0));
  }
  c->last_launches = c->launches_per_iter;
  for (int i = 0; i < n_iters; ++i) CK(cudaGraphLaunch(c->graph_exec, c->stream));
  c->iters_run += n_iters;
  return NMF_OK;
}

// Comparator forms of one iteration (same products and objective as
// enq_iteration, other updates; same entry/exit invariant: S = W^T W and
// R = A^T W for the current W):
//   FORM_ALG1: Alg. 1 as written, the updates column by column (alg1.cu);
//   FORM_MU:   multiplicative updates (mu.cu), H then W.
enum AltForm { FORM_ALG1 = 0, FORM_MU = 1 };

cudaError_t enq_update_alt(nmf_ctx* c, AltForm f, bool is_w, cudaStream_t s, int* launches) {
  if (f == FORM_ALG1)
    return is_w ? alg1_update_w(c->W, c->P, c->Q, c->V, c->K, c->Kp, c->eps, c->alg1_part, c->d_status, s, launches)
                : alg1_update_h(c->Ht, c->R, c->S, c->D, c->K, c->Kp, c->eps, s, launches);
  return is_w ? mu_update(c->W, c->P, c->Q, c->Y, c->V, c->K, c->Kp, c->eps, s, launches)
              : mu_update(c->Ht, c->R, c->S, c->Y, c->D, c->K, c->Kp, c->eps, s, launches);
}

cudaError_t enq_alt_iteration(nmf_ctx* c, AltForm f) {
  cudaError_t e;
  if ((e = enq_update_alt(c, f, false, c->stream, &c->launch_count)) != cudaSuccess) return e;
  if ((e = enq_product_P(c)) != cudaSuccess) return e;
  if ((e = enq_gram(c, c->gramH, c->Ht, c->Q)) != cudaSuccess) return e;
  if ((e = enq_update_alt(c, f, true, c->stream, &c->launch_count)) != cudaSuccess) return e;
  if ((e = enq_product_R(c)) != cudaSuccess) return e;
  if ((e = enq_gram(c, c->gramW, c->W, c->S)) != cudaSuccess) return e;
  return enq_objective(c);
}

nmf_status iterate_alt(nmf_ctx* c, AltForm f, int32_t n_iters, float* step_ms) {
  if (!c || n_iters < 0) return NMF_EINVAL;
  if (n_iters == 0) return NMF_OK;
  CK(ensure_entry(c));
  if (step_ms) {
    // Steps in NMF_PROFILE_STEPS order: 0 R, 1 H, 2 P, 3 Q, 4 W, 5 S, 6 objective.
    cudaEvent_t ev[8];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    double acc[NMF_PROFILE_STEPS] = {0};
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < n_iters && e == cudaSuccess; ++it) {
      cudaStream_t s = c->stream;
      e = cudaEventRecord(ev[0], s);                                           // H
      if (e == cudaSuccess) e = enq_update_alt(c, f, false, s, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);                     // P
      if (e == cudaSuccess) e = enq_product_P(c);
      if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);                     // Q
      if (e == cudaSuccess) e = enq_gram(c, c->gramH, c->Ht, c->Q);
      if (e == cudaSuccess) e = cudaEventRecord(ev[3], s);                     // W
      if (e == cudaSuccess) e = enq_update_alt(c, f, true, s, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(ev[4], s);                     // R
      if (e == cudaSuccess) e = enq_product_R(c);
      if (e == cudaSuccess) e = cudaEventRecord(ev[5], s);                     // S
      if (e == cudaSuccess) e = enq_gram(c, c->gramW, c->W, c->S);
      if (e == cudaSuccess) e = cudaEventRecord(ev[6], s);                     // objective
      if (e == cudaSuccess) e = enq_objective(c);
      if (e == cudaSuccess) e = cudaEventRecord(ev[7], s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[7]);
      const int slot[7] = {1, 2, 3, 4, 0, 5, 6};
      for (int k = 0; k < 7 && e == cudaSuccess; ++k) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
        acc[slot[k]] += ms;
      }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    CK(e);
    for (int k = 0; k < NMF_PROFILE_STEPS; ++k) step_ms[k] = (float)(acc[k] / n_iters);
    c->iters_run += n_iters;
    return read_status(c);
  }
  cudaGraph_t& graph = f == FORM_ALG1 ? c->graph_alg1 : c->graph_mu;
  cudaGraphExec_t& exec = f == FORM_ALG1 ? c->graph_alg1_exec : c->graph_mu_exec;
  if (!exec) {
    c->launch_count = 0;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enq_alt_iteration(c, f);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return from_cuda(e != cudaSuccess ? e : e2);
    }
    graph = g;
    (f == FORM_ALG1 ? c->launches_alg1 : c->launches_mu) = c->launch_count;
    CK(cudaGraphInstantiate(&exec, g, 0));
  }
  c->last_launches = f == FORM_ALG1 ? c->launches_alg1 : c->launches_mu;
  for (int i = 0; i < n_iters; ++i) CK(cudaGraphLaunch(exec, c->stream));
  c->iters_run += n_iters;
  return NMF_OK;
}

nmf_status nmf_iterate_alg1(nmf_ctx* c, int32_t n_iters, float* step_ms) {
  return iterate_alt(c, FORM_ALG1, n_iters, step_ms);
}

nmf_status nmf_iterate_mu(nmf_ctx* c, int32_t n_iters, float* step_ms) {
  return iterate_alt(c, FORM_MU, n_iters, step_ms);
}

nmf_status nmf_warm_h(nmf_ctx* c, nmf_mlp* mlp, const nmf_problem* nd, float tol, int32_t max_sweeps,
                      const float* H_ref, float* H_out, float* R_out, int32_t* sweeps_out, double* trace) {
  if (!c || !nd || !H_out || max_sweeps < 0 || !(tol >= 0.f)) return NMF_EINVAL;
  if (nd->fmt != NMF_CSR_F32_I32 || nd->V != c->V || nd->K != c->K || nd->D < 1) return NMF_EINVAL;
  if (mlp && mlp_K(mlp) != c->K) return NMF_EINVAL;
  const int V = c->V, N = nd->D, K = c->K, Kp = c->Kp;
  cudaStream_t s = c->stream;
  std::vector<int> rp, ci;
  std::vector<float> va;
  double normA2 = 0.0;
  nmf_status st = validate_and_copy_csr(nd, rp, ci, va, &normA2);
  if (st != NMF_OK) return st;
  // CSR of A_new^T (documents as rows), stable counting sort.
  const int64_t nnz = nd->nnz;
  std::vector<int> rpT((size_t)N + 1, 0), ciT((size_t)nnz);
  std::vector<float> vaT((size_t)nnz);
  for (int64_t e = 0; e < nnz; ++e) rpT[(size_t)ci[e] + 1]++;
  for (int d = 0; d < N; ++d) rpT[d + 1] += rpT[d];
  {
    std::vector<int> fill(rpT.begin(), rpT.end() - 1);
    for (int r = 0; r < V; ++r)
      for (int e = rp[r]; e < rp[r + 1]; ++e) {
        const int pos = fill[ci[e]]++;
        ciT[pos] = r;
        vaT[pos] = va[e];
      }
  }
  int* d_ciT = nullptr;
  float* d_vaT = nullptr;
  float *Rn = nullptr, *Hn = nullptr, *Hp = nullptr, *Hr = nullptr, *tmp = nullptr;
  double* part = nullptr;
  double* d_trace = nullptr;
  int* d_state = nullptr;
  SpmmPlan plan;
  auto cleanup = [&](nmf_status r) {
    cudaStreamSynchronize(s);
    spmm_plan_free(plan);
    for (void* q : {(void*)d_ciT, (void*)d_vaT, (void*)Rn, (void*)Hn, (void*)Hp, (void*)Hr, (void*)tmp, (void*)part,
                    (void*)d_trace, (void*)d_state})
      if (q) cudaFree(q);
    return r;
  };
#define WK(x)                                     \
  do {                                            \
    const cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) {                      \
      cudaGetLastError();                         \
      return cleanup(from_cuda(e_));              \
    }                                             \
  } while (0)
  const size_t nk = (size_t)N * Kp;
  WK(cudaMalloc(&d_ciT, sizeof(int) * std::max<size_t>(1, ciT.size())));
  WK(cudaMalloc(&d_vaT, sizeof(float) * std::max<size_t>(1, vaT.size())));
  if (nnz > 0) {
    WK(cudaMemcpy(d_ciT, ciT.data(), sizeof(int) * ciT.size(), cudaMemcpyHostToDevice));
    WK(cudaMemcpy(d_vaT, vaT.data(), sizeof(float) * vaT.size(), cudaMemcpyHostToDevice));
  }
  WK(spmm_plan_build(plan, rpT, N, V, Kp, 512));
  WK(cudaMalloc(&Rn, sizeof(float) * nk));
  WK(cudaMalloc(&Hn, sizeof(float) * nk));
  WK(cudaMalloc(&tmp, sizeof(float) * std::max(nk, (size_t)K * N)));
  WK(cudaMalloc(&part, sizeof(double) * std::max(diff_norm_partials(), h_sweep_partials(N))));
  WK(cudaMemsetAsync(Hn, 0, sizeof(float) * nk, s));
  if (H_ref) {
    WK(cudaMalloc(&Hr, sizeof(float) * nk));
    WK(cudaMemcpyAsync(tmp, H_ref, sizeof(float) * (size_t)K * N, cudaMemcpyDefault, s));
    WK(cudaMemsetAsync(Hr, 0, sizeof(float) * nk, s));
    WK(transpose_f32(tmp, K, N, N, Hr, Kp, s));
  } else if ((Kp + 31) / 32 == 1) {
    WK(cudaMalloc(&Hp, sizeof(float) * nk));              // the previous sweep's H (row-per-warp form)
  }
  // S = W^T W of the fixed W; R = A_new^T W.
  if (!c->s_valid) {
    WK(enq_gram(c, c->gramW, c->W, c->S));
    c->s_valid = true;
  }
  WK(spmm_run(plan, d_ciT, d_vaT, c->W, Rn, Kp, s));
  if (R_out) WK(cudaMemcpy2DAsync(R_out, sizeof(float) * K, Rn, sizeof(float) * Kp, sizeof(float) * K, N,
                                  cudaMemcpyDefault, s));
  if (mlp) {
    WK(mlp_forward_dev(mlp, Rn, Kp, N, Hn, Kp, s));
  } else {
    WK(fill_uniform_splitmix_t(Hn, N, K, Kp, nd->seed ^ 0x4848484848484848ull, s));
  }
  // Sweeps enqueued kSweepChunk at a time; each sweep's check runs on the
  // device (diff_check), and once it has met tol the later sweeps of the
  // chunk leave H as it is, so the host reads the state back once per chunk.
  constexpr int kSweepChunk = 32;
  WK(cudaMalloc(&d_state, sizeof(int) * 2));
  WK(cudaMalloc(&d_trace, sizeof(double) * std::max(1, max_sweeps)));
  WK(cudaMemsetAsync(d_state, 0, sizeof(int) * 2, s));
  int done = 0;
  for (int sw0 = 1; sw0 <= max_sweeps; sw0 += kSweepChunk) {
    const int sw1 = std::min(max_sweeps, sw0 + kSweepChunk - 1);
    for (int sw = sw0; sw <= sw1; ++sw)
      WK(h_update_sweep(Hn, Rn, c->S, N, K, Kp, c->eps, c->d_status, s, H_ref ? Hr : nullptr, Hp, part, tol, sw,
                        d_trace, d_state));
    int st[2] = {0, 0};
    WK(cudaMemcpyAsync(st, d_state, sizeof(st), cudaMemcpyDeviceToHost, s));
    WK(cudaStreamSynchronize(s));
    done = st[1];
    if (st[0]) break;
  }
  if (trace && done > 0) WK(cudaMemcpyAsync(trace, d_trace, sizeof(double) * done, cudaMemcpyDeviceToHost, s));
  WK(transpose_f32(Hn, N, K, Kp, tmp, N, s));
  WK(cudaMemcpyAsync(H_out, tmp, sizeof(float) * (size_t)K * N, cudaMemcpyDefault, s));
  WK(cudaStreamSynchronize(s));
#undef WK
  if (sweeps_out) *sweeps_out = done;
  const nmf_status rs = read_status(c);
  return cleanup(rs);
}

nmf_status nmf_error(nmf_ctx* c, double* frob2, double* rel) {
  if (!c) return NMF_EINVAL;
  if (c->iters_run == 0) {
    // Objective of the initial factors.
    c->launch_count = 0;
    CK(enq_product_P(c));
    CK(enq_gram(c, c->gramH, c->Ht, c->Q));
    CK(enq_gram(c, c->gramW, c->W, c->S));
    CK(enq_objective(c));
    c->s_valid = true;
  }
  double f = NAN;
  if (c->fmt == NMF_DENSE_F32) {
    // Dense A: Eq. 2 evaluated directly, sum of (A - WH)^2 accumulated in
    // FP64 from the FP32 A (no cancellation; in the BF16 form this measures
    // the fit to A itself rather than to its BF16 copy).
    CK(resid2_dense(c->dense, c->lda, c->W, c->Ht, c->V, c->D, c->K, c->Kp, c->resid_part, &f, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  nmf_status st = read_status(c);
  unsigned cnt = 0;
  CK(cudaMemcpy(&cnt, c->d_counter, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (c->fmt != NMF_DENSE_F32 && cnt > 0)
    CK(cudaMemcpy(&f, c->hist + (cnt - 1) % kHistCap, sizeof(double), cudaMemcpyDeviceToHost));
  if (frob2) *frob2 = f;
  if (rel) *rel = std::sqrt(std::max(f, 0.0) / c->normA2);
  return st;
}

nmf_status nmf_objective_history(nmf_ctx* c, double* out, int32_t n) {
  if (!c || !out || n < 0 || n > kHistCap) return NMF_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  unsigned cnt = 0;
  CK(cudaMemcpy(&cnt, c->d_counter, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if ((unsigned)n > cnt) return NMF_EINVAL;
  std::vector<double> h(kHistCap);
  CK(cudaMemcpy(h.data(), c->hist, sizeof(double) * kHistCap, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) out[i] = h[(cnt - n + i) % kHistCap];
  return read_status(c);
}

// One iteration on host-held factors.  With host buffers the runtime can
// copy asynchronously (pinned, or device memory) the copies are captured
// with the iteration into one graph (cached for the last pointer set):
//   main:  W_in -> W | R = A^T W | (S, H_in landed) H update | P | W update | S, objective | objective -> host
//   side2:            S = W^T W                                                <W, P>
//   side3:            H_in -> stage -> H^T   H^T -> stage -> H_out    W -> W_out
// W comes in first, at the link's full rate, since R and S need it; H's copy
// in then runs beside R and S, its copy out beside P, Q and the W update,
// and W's copy out beside S and the objective.  The status word comes back
// with the outputs.  Other host memory is copied before and after one
// nmf_iterate, without overlap.
nmf_status nmf_iterate_host(nmf_ctx* c, const float* W_in, const float* H_in, float* W_out, float* H_out,
                            double* frob2) {
  if (!c) return NMF_EINVAL;
  auto async_ok = [](const void* p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice;
  };
  const bool dense = c->fmt == NMF_DENSE_F32;
  if (!async_ok(W_in) || !async_ok(H_in) || !async_ok(W_out) || !async_ok(H_out)) {
    nmf_status st = nmf_set_factors(c, W_in, H_in);
    if (st != NMF_OK) return st;
    if ((st = nmf_iterate(c, 1)) != NMF_OK) return st;
    double f = 0.0;
    if (frob2 && (st = nmf_error(c, &f, nullptr)) != NMF_OK) return st;
    if (frob2) *frob2 = f;
    return nmf_get_factors(c, W_out, H_out);
  }
  const void* key[5] = {W_in, H_in, W_out, H_out, (frob2 && !dense) ? c : nullptr};
  if (c->graph_io_exec && std::memcmp(key, c->io_key, sizeof(key)) != 0) {
    cudaGraphExecDestroy(c->graph_io_exec);
    cudaGraphDestroy(c->graph_io);
    c->graph_io_exec = nullptr;
    c->graph_io = nullptr;
  }
  if (!c->graph_io_exec) {
    cudaStream_t m = c->stream;
    const int K = c->K, Kp = c->Kp;
    c->launch_count = 0;
    CK(cudaStreamBeginCapture(m, cudaStreamCaptureModeThreadLocal));
    auto body = [&]() -> cudaError_t {
      cudaError_t e;
      // W first at the link's full rate (R and S wait for it), then H while
      // they run.
      if (W_in && (e = cudaMemcpy2DAsync(c->W, sizeof(float) * Kp, W_in, sizeof(float) * K, sizeof(float) * K, c->V,
                                         cudaMemcpyDefault, m)) != cudaSuccess)
        return e;
      if ((e = cudaEventRecord(c->evio[2], m)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(c->side3, c->evio[2], 0)) != cudaSuccess) return e;
      if (H_in) {
        if ((e = cudaMemcpyAsync(c->stage, H_in, sizeof(float) * (size_t)K * c->D, cudaMemcpyDefault, c->side3)) !=
            cudaSuccess)
          return e;
        c->launch_count += 1;
        if ((e = transpose_f32(c->stage, K, c->D, c->D, c->Ht, Kp, c->side3)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->evio[3], c->side3)) != cudaSuccess) return e;
      }
      // Entry state of the iteration for this W: S beside R (in the BF16
      // form both read one BF16 operand of W, made first).
      const bool shared_op = c->bf16 && c->tma;
      if (shared_op && (e = bf16_operand(c, true, m)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(c->evio[4], m)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(c->side2, c->evio[4], 0)) != cudaSuccess) return e;
      if ((e = enq_gram(c, c->gramW, c->W, c->S, c->side2, shared_op)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(c->evio[5], c->side2)) != cudaSuccess) return e;
      if ((e = enq_product_R(c, m, shared_op)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(m, c->evio[5], 0)) != cudaSuccess) return e;
      if (H_in && (e = cudaStreamWaitEvent(m, c->evio[3], 0)) != cudaSuccess) return e;
      IoHooks io;
      io.H_out = H_out;
      io.W_out = W_out;
      io.obj_host = key[4] ? c->h_obj : nullptr;
      if ((e = enq_iteration(c, &io)) != cudaSuccess) return e;
      return cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, m);
    };
    const cudaError_t e = body();
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(m, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return from_cuda(e != cudaSuccess ? e : e2);
    }
    c->graph_io = g;
    const cudaError_t e3 = cudaGraphInstantiate(&c->graph_io_exec, g, 0);
    if (e3 != cudaSuccess) {
      cudaGraphDestroy(g);
      c->graph_io = nullptr;
      c->graph_io_exec = nullptr;
      return from_cuda(e3);
    }
    std::memcpy(c->io_key, key, sizeof(key));
  }
  CK(cudaGraphLaunch(c->graph_io_exec, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->iters_run += 1;
  c->s_valid = true;      // S of the new W was formed for the objective
  c->r_valid = false;     // R of the new W was not
  if (*c->h_status != 0) {
    nmf_status st = read_status(c);       // reports and clears it
    if (st != NMF_OK) return st;
  }
  if (frob2) {
    if (dense) return nmf_error(c, frob2, nullptr);
    *frob2 = *c->h_obj;
  }
  return NMF_OK;
}

nmf_status nmf_get_factors(nmf_ctx* c, float* W, float* H) {
  if (!c) return NMF_EINVAL;
  const int K = c->K, Kp = c->Kp;
  if (W)
    CK(cudaMemcpy2DAsync(W, sizeof(float) * K, c->W, sizeof(float) * Kp, sizeof(float) * K, c->V,
                         cudaMemcpyDefault, c->stream));
  if (H) {
    CK(transpose_f32(c->Ht, c->D, K, Kp, c->stage, c->D, c->stream));
    CK(cudaMemcpyAsync(H, c->stage, sizeof(float) * (size_t)K * c->D, cudaMemcpyDefault, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return read_status(c);
}

nmf_status nmf_set_factors(nmf_ctx* c, const float* W, const float* H) {
  if (!c) return NMF_EINVAL;
  const int K = c->K, Kp = c->Kp;
  if (W) {
    CK(cudaMemcpy2DAsync(c->W, sizeof(float) * Kp, W, sizeof(float) * K, sizeof(float) * K, c->V,
                         cudaMemcpyDefault, c->stream));
    c->s_valid = false;
    c->r_valid = false;
  }
  if (H) {
    CK(cudaMemcpyAsync(c->stage, H, sizeof(float) * (size_t)K * c->D, cudaMemcpyDefault, c->stream));
    CK(transpose_f32(c->stage, K, c->D, c->D, c->Ht, Kp, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return NMF_OK;
}

nmf_status nmf_run_step(nmf_ctx* c, int32_t step) {
  if (!c) return NMF_EINVAL;
  c->launch_count = 0;
  switch (step) {
    case NMF_STEP_R: CK(enq_product_R(c)); c->r_valid = true; break;
    case NMF_STEP_S: CK(enq_gram(c, c->gramW, c->W, c->S)); c->s_valid = true; break;
    case NMF_STEP_UPDATE_H: CK(enq_update(c, c->Ht, c->S, c->R, c->D, false)); break;
    case NMF_STEP_P: CK(enq_product_P(c)); break;
    case NMF_STEP_Q: CK(enq_gram(c, c->gramH, c->Ht, c->Q)); break;
    case NMF_STEP_UPDATE_W:
      CK(enq_update(c, c->W, c->Q, c->P, c->V, true));
      c->s_valid = false;
      c->r_valid = false;
      break;
    case NMF_STEP_OBJECTIVE:
      CK(enq_gram(c, c->gramW, c->W, c->S));
      c->s_valid = true;
      CK(enq_objective(c));
      break;
    default: return NMF_EINVAL;
  }
  return NMF_OK;
}

nmf_status nmf_get_buffer(nmf_ctx* c, int32_t which, float* dst, int64_t count) {
  if (!c || !dst) return NMF_EINVAL;
  const int K = c->K, Kp = c->Kp;
  const float* src = nullptr;
  int rows = 0;
  switch (which) {
    case NMF_BUF_W: src = c->W; rows = c->V; break;
    case NMF_BUF_HT: src = c->Ht; rows = c->D; break;
    case NMF_BUF_R: src = c->R; rows = c->D; break;
    case NMF_BUF_P: src = c->P; rows = c->V; break;
    case NMF_BUF_S: src = c->S; rows = K; break;
    case NMF_BUF_Q: src = c->Q; rows = K; break;
    default: return NMF_EINVAL;
  }
  if (count != (int64_t)rows * K) return NMF_EINVAL;
  CK(cudaMemcpy2DAsync(dst, sizeof(float) * K, src, sizeof(float) * Kp, sizeof(float) * K, rows,
                       cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return read_status(c);
}

nmf_status nmf_set_buffer(nmf_ctx* c, int32_t which, const float* src, int64_t count) {
  if (!c || !src) return NMF_EINVAL;
  const int K = c->K, Kp = c->Kp;
  float* dst = nullptr;
  int rows = 0;
  switch (which) {
    case NMF_BUF_W: dst = c->W; rows = c->V; c->s_valid = false; c->r_valid = false; break;
    case NMF_BUF_HT: dst = c->Ht; rows = c->D; break;
    case NMF_BUF_R: dst = c->R; rows = c->D; c->r_valid = false; break;
    case NMF_BUF_P: dst = c->P; rows = c->V; break;
    case NMF_BUF_S: dst = c->S; rows = K; c->s_valid = false; break;
    case NMF_BUF_Q: dst = c->Q; rows = K; break;
    default: return NMF_EINVAL;
  }
  if (count != (int64_t)rows * K) return NMF_EINVAL;
  CK(cudaMemcpy2DAsync(dst, sizeof(float) * Kp, src, sizeof(float) * K, sizeof(float) * K, rows,
                       cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return NMF_OK;
}

nmf_status nmf_profile(nmf_ctx* c, int32_t n_iters, float* step_ms) {
  if (!c || !step_ms || n_iters <= 0) return NMF_EINVAL;
  if (!c->s_valid) {
    CK(enq_gram(c, c->gramW, c->W, c->S));
    c->s_valid = true;
  }
  cudaEvent_t ev[NMF_PROFILE_STEPS + 1];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  double acc[NMF_PROFILE_STEPS] = {0};
  nmf_status st = NMF_OK;
  for (int it = 0; it < n_iters && st == NMF_OK; ++it) {
    cudaError_t e = cudaSuccess;
    e = cudaEventRecord(ev[0], c->stream);
    if (e == cudaSuccess) e = enq_product_R(c);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
    if (e == cudaSuccess) e = enq_update(c, c->Ht, c->S, c->R, c->D, false);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->stream);
    if (e == cudaSuccess) e = enq_product_P(c);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], c->stream);
    if (e == cudaSuccess) e = enq_gram(c, c->gramH, c->Ht, c->Q);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4], c->stream);
    if (e == cudaSuccess) e = enq_update(c, c->W, c->Q, c->P, c->V, true, false, true);
    if (e == cudaSuccess) e = cudaEventRecord(ev[5], c->stream);
    if (e == cudaSuccess) e = enq_gram_after_w(c, nullptr, false);
    if (e == cudaSuccess) e = cudaEventRecord(ev[6], c->stream);
    if (e == cudaSuccess) e = enq_objective(c);
    if (e == cudaSuccess) e = cudaEventRecord(ev[7], c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[7]);
    for (int k = 0; k < NMF_PROFILE_STEPS && e == cudaSuccess; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      acc[k] += ms;
    }
    st = from_cuda(e);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  c->s_valid = true;          // S of the new W was the last product formed
  c->r_valid = false;         // R was formed from the W before the update
  if (st != NMF_OK) return st;
  c->iters_run += n_iters;
  for (int k = 0; k < NMF_PROFILE_STEPS; ++k) step_ms[k] = (float)(acc[k] / n_iters);
  return read_status(c);
}

nmf_status nmf_query(nmf_ctx* c, int32_t* tile_T, int32_t* chain_ctas, int32_t* launches_per_iter) {
  if (!c) return NMF_EINVAL;
  if (chain_ctas && c->w_persistent) {
    *chain_ctas = c->wp.cluster;
    if (tile_T) *tile_T = c->T;
    if (launches_per_iter) *launches_per_iter = c->last_launches ? c->last_launches : c->launches_per_iter;
    return NMF_OK;
  }
  if (tile_T) *tile_T = c->T;
  if (chain_ctas) *chain_ctas = c->chainW.cluster;
  if (launches_per_iter) *launches_per_iter = c->last_launches ? c->last_launches : c->launches_per_iter;
  return NMF_OK;
}

nmf_status nmf_query_form(nmf_ctx* c, int32_t* w_single_launch, int32_t* s_in_w_update, int32_t* s_chunks) {
  if (!c) return NMF_EINVAL;
  if (w_single_launch) *w_single_launch = c->w_persistent ? 1 : 0;
  if (s_in_w_update) *s_in_w_update = c->ws_gram ? 1 : 0;
  if (s_chunks) *s_chunks = c->ws_gram ? c->gramW.n_chunks : 0;
  return NMF_OK;
}

nmf_status nmf_set_spmm_split(nmf_ctx* c, int32_t seg_P, int32_t seg_R) {
  if (!c || seg_P < 0 || seg_R < 0 || (seg_P > 0 && seg_P < 16) || (seg_R > 0 && seg_R < 16)) return NMF_EINVAL;
  if (c->fmt != NMF_CSR_F32_I32) return NMF_EUNSUPPORTED;
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);                       // the captured launches name the old plans' arrays
  CK(set_spmm_seg(c, 0, seg_P ? seg_P : kNoSplit));
  CK(set_spmm_seg(c, 1, seg_R ? seg_R : kNoSplit));
  c->r_valid = false;                  // R of the old plan: recomputed with the new one
  return NMF_OK;
}

nmf_status nmf_tune_spmm(nmf_ctx* c, int32_t* seg_P, int32_t* seg_R) {
  if (!c) return NMF_EINVAL;
  if (c->fmt != NMF_CSR_F32_I32) return NMF_EUNSUPPORTED;
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  c->r_valid = false;
  CK(tune_spmm_segs(c));
  CK(cudaStreamSynchronize(c->stream));
  c->r_valid = true;                   // formed with the chosen plan for the current W
  if (seg_P) *seg_P = c->segA == kNoSplit ? 0 : c->segA;
  if (seg_R) *seg_R = c->segAt == kNoSplit ? 0 : c->segAt;
  return NMF_OK;
}

nmf_status nmf_set_w_workers_after_chain(nmf_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return NMF_EINVAL;
  if (!c->w_persistent) return NMF_EUNSUPPORTED;
  c->w_workers_after_chain = on != 0;
  drop_graph(c);
  return NMF_OK;
}

nmf_status nmf_set_wait_limits(nmf_ctx* c, int64_t wait_ns, int32_t extra_arrivals) {
  if (!c || wait_ns < 0 || extra_arrivals < 0) return NMF_EINVAL;
  if (!c->w_persistent) return NMF_EUNSUPPORTED;
  c->wait_ns = (unsigned long long)wait_ns;
  c->extra_arrivals = extra_arrivals;
  drop_graph(c);
  return NMF_OK;
}

void nmf_destroy(nmf_ctx* c) { free_ctx(c); }

nmf_status nmf_gemm(int32_t M, int32_t N, int32_t K, const float* A, int64_t lda, int32_t transA,
                    const float* B, int64_t ldb, float* C, int64_t ldc, int32_t prec, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return NMF_EINVAL;
  if (prec != NMF_PREC_FP32 && prec != NMF_PREC_BF16) return NMF_EINVAL;
  static int* d_status = nullptr;
  if (!d_status) {
    CK(cudaMalloc(&d_status, sizeof(int)));
    CK(cudaMemset(d_status, 0, sizeof(int)));
  }
  GemmArgs g;
  g.M = M; g.N = N; g.Kin = K;
  g.A = A; g.lda = lda; g.transA = transA ? 1 : 0;
  g.B = B; g.ldb = ldb;
  g.C = C; g.ldc = ldc;
  g.mode = GM_STORE;
  return from_cuda(tc_gemm_run(g, prec == NMF_PREC_FP32 ? TC_TF32X3 : TC_BF16, nullptr, 0, d_status,
                               static_cast<cudaStream_t>(stream)));
}

nmf_status nmf_gemm_bf16(int32_t M, int32_t N, int32_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                         int64_t ldb, float* C, int64_t ldc, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || lda < K || ldb < K || ldc < N) return NMF_EINVAL;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) || (lda & 7) || (ldb & 7))
    return NMF_EINVAL;
  if (!tma_available()) return NMF_EUNSUPPORTED;
  static int* d_status = nullptr;
  if (!d_status) {
    CK(cudaMalloc(&d_status, sizeof(int)));
    CK(cudaMemset(d_status, 0, sizeof(int)));
  }
  return from_cuda(tc_bf16_tma_gemm(A, lda, B, ldb, C, ldc, M, N, K, d_status, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
