"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the
same seeded inputs.  Tolerances (FP32 path): after one iteration the
max-norm relative difference of W and of H is at most 1e-5; after the full
iteration count the objective (Eq. 2, evaluated by the oracle in FP64 on the
GPU's factors) is within 1e-4 relative of the oracle's own run."""

import math

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle import objective as ob
from paper_1904_07935_b300 import synth

from ._parity import (colmax_rel, f32, forward_error_ratio, fp32_storage_sensitivity, h_update_scale,
                      rel_h, rel_w)

pytestmark = pytest.mark.gpu

EPS = 1e-16
TOL_ITER = 1e-5      # one iteration, FP32 path
TOL_OBJ = 1e-4       # relative objective after the full run, FP32 path


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


def _dense_ctx(nmf, A, K, W0, H0, **kw):
    import torch
    return nmf.from_dense(A, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(), **kw)


def _sparse_ctx(nmf, prob, K, W0, H0, **kw):
    import torch
    return nmf.from_sparse(prob, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(), **kw)


def _oracle_start(W0, H0):
    """The oracle's view of the initial factors: W with unit columns (FP64)."""
    return fh.normalize_init(W0), H0.astype(np.float64)


# --- initialisation -----------------------------------------------------------

def test_device_init_matches_splitmix_definition(nmf):
    prob = synth.planted_dense(96, 80, 4, 3)
    ctx = nmf.from_dense(prob.A, 7, seed=1234)
    W, H = ctx.get_factors()
    W0, H0 = synth.init_factors(1234, 96, 80, 7)
    assert np.array_equal(H, H0)                               # bit-exact draws
    Wn = W0.astype(np.float64) / np.linalg.norm(W0.astype(np.float64), axis=0)
    assert np.max(np.abs(W - Wn)) < 2e-7
    assert np.allclose(np.linalg.norm(W.astype(np.float64), axis=0), 1.0, atol=1e-6)


# --- products and Grams -------------------------------------------------------

def _check_products(ctx, nmf, A64, W, H, tol):
    ctx.set_buffer(nmf.BUF_W, W)
    ctx.set_buffer(nmf.BUF_HT, np.ascontiguousarray(H.T))
    for st in (nmf.STEP_R, nmf.STEP_S, nmf.STEP_P, nmf.STEP_Q):
        ctx.run_step(st)
    W64, H64 = W.astype(np.float64), H.astype(np.float64)
    R = np.asarray(A64.T @ W64)
    P = np.asarray(A64 @ H64.T)
    for which, ref in ((nmf.BUF_R, R), (nmf.BUF_P, P), (nmf.BUF_S, W64.T @ W64), (nmf.BUF_Q, H64 @ H64.T)):
        got = ctx.get_buffer(which)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < tol, (which, err)


def test_dense_products_and_grams(nmf):
    prob = synth.planted_dense(300, 230, 5, 11)             # ragged vs the 64-wide tiles
    W0, H0 = synth.init_factors(12, 300, 230, 13)          # K = 13: padded to 16
    ctx = _dense_ctx(nmf, prob.A, 13, W0, H0)
    _check_products(ctx, nmf, prob.A.astype(np.float64), W0, H0, 2e-6)


@pytest.mark.parametrize("K", [37, 100, 176, 320])
def test_sparse_products_with_long_and_empty_rows(nmf, K):
    sp = synth.sparse_termdoc(3000, 1400, 21, mean_terms=40)
    lens = np.diff(sp.A.row_ptr)
    assert lens.max() > 512 and (lens == 0).any()          # split rows and empty rows
    W0, H0 = synth.init_factors(22, 3000, 1400, K)
    ctx = _sparse_ctx(nmf, sp, K, W0, H0)
    _check_products(ctx, nmf, sp.A.to_scipy().astype(np.float64), W0, H0, 3e-6)


@pytest.mark.parametrize("seg", [0, 16, 100, 256, 1024])
def test_sparse_products_at_every_split_length(nmf, seg):
    """R and P with long rows cut into pieces of `seg` non-zeros (0: no
    split): the same products up to rounding for every schedule."""
    sp = synth.sparse_termdoc(3000, 1400, 23, mean_terms=40)
    assert np.diff(sp.A.row_ptr).max() > 1024
    W0, H0 = synth.init_factors(24, 3000, 1400, 100)
    ctx = _sparse_ctx(nmf, sp, 100, W0, H0)
    ctx.set_spmm_split(seg, seg)
    _check_products(ctx, nmf, sp.A.to_scipy().astype(np.float64), W0, H0, 3e-6)


def test_tuned_split_is_reproduced_by_setting_it(nmf):
    """nmf_tune_spmm picks lengths from its candidate set, keeps R valid
    for the current W, and a context given the same lengths by
    nmf_set_spmm_split iterates bit-identically; the iteration stays within
    the one-iteration tolerance of the oracle."""
    K = 64
    sp = synth.sparse_termdoc(6000, 2500, 25, mean_terms=60)
    W0, H0 = synth.init_factors(26, 6000, 2500, K)
    tuned = _sparse_ctx(nmf, sp, K, W0, H0)
    segP, segR = tuned.tune_spmm()
    assert segP in (128, 256, 512, 1024, 0) and segR in (128, 256, 512, 1024, 0)
    tuned.iterate(2)
    fixed = _sparse_ctx(nmf, sp, K, W0, H0)
    fixed.set_spmm_split(segP, segR)
    fixed.iterate(2)
    Wt, Ht = tuned.get_factors()
    Wf, Hf = fixed.get_factors()
    assert np.array_equal(Wt, Wf) and np.array_equal(Ht, Hf)
    one = _sparse_ctx(nmf, sp, K, W0, H0)
    one.set_spmm_split(segP, segR)
    one.iterate(1)
    Wg, Hg = one.get_factors()
    Wr, Hr = _oracle_start(W0, H0)
    Wr, Hr = fh.iteration(sp.A, Wr, Hr)
    assert rel_w(Wg, Wr) < TOL_ITER and rel_h(Hg, Hr) < TOL_ITER


def test_spmm_split_rejects_bad_arguments(nmf):
    sp = synth.sparse_termdoc(2000, 900, 27, mean_terms=30)
    ctx = nmf.from_sparse(sp, 16)
    for a, b in ((-1, 512), (512, 8), (1, 1)):
        with pytest.raises(nmf.NmfError) as e:
            ctx.set_spmm_split(a, b)
        assert e.value.status == nmf.NMF_EINVAL
    prob = synth.planted_dense(100, 80, 4, 3)
    dense = nmf.from_dense(prob.A, 8)
    for call in (lambda: dense.set_spmm_split(512, 512), dense.tune_spmm):
        with pytest.raises(nmf.NmfError) as e:
            call()
        assert e.value.status == nmf.NMF_EUNSUPPORTED


# --- factor updates in isolation ----------------------------------------------

@pytest.mark.parametrize("K,T", [(16, 16), (16, 1), (20, 3), (37, 16), (48, 8)])
def test_update_h_matches_alg1(nmf, K, T):
    prob = synth.planted_dense(260, 700, 6, 31)
    W0, H0 = synth.init_factors(32 + K, 260, 700, K)
    W, H = _oracle_start(W0, H0)
    A = prob.A.astype(np.float64)
    R, S = f32(A.T @ W), f32(W.T @ W)
    Hin = f32(H)
    ctx = _dense_ctx(nmf, prob.A, K, W0, H0, tile_T=T)
    ctx.set_buffer(nmf.BUF_R, R)
    ctx.set_buffer(nmf.BUF_S, S)
    ctx.set_buffer(nmf.BUF_HT, np.ascontiguousarray(Hin.T))
    ctx.run_step(nmf.STEP_UPDATE_H)
    got = ctx.get_buffer(nmf.BUF_HT).T
    ref = fh.update_h(R.astype(np.float64), S.astype(np.float64), Hin, EPS)
    assert rel_h(got, ref) < TOL_ITER
    # kernel arithmetic: error within FP32 rounding of the terms it combines
    assert forward_error_ratio(got, ref, h_update_scale(R, S, Hin, ref)) < 1e-6


@pytest.mark.parametrize("K,D", [(64, 1500), (160, 11314), (176, 3001), (37, 149)])
def test_update_h_row_counts_and_wide_ranks(nmf, K, D):
    """The H update alone at the text-like document count (11,314 rows, one
    row per group of four lanes), at K = 176 (11 tiles, S's blocks fetched
    tile by tile) and on 149 rows with K = 37 (fewer rows than SMs, a ragged
    last block of the off-tile sums)."""
    V = 300
    prob = synth.planted_dense(V, D, 6, 53 + K)
    W0, H0 = synth.init_factors(54 + K, V, D, K)
    W, H = _oracle_start(W0, H0)
    A = prob.A.astype(np.float64)
    R, S = f32(A.T @ W), f32(W.T @ W)
    Hin = f32(H)
    ctx = _dense_ctx(nmf, prob.A, K, W0, H0)
    ctx.set_buffer(nmf.BUF_R, R)
    ctx.set_buffer(nmf.BUF_S, S)
    ctx.set_buffer(nmf.BUF_HT, np.ascontiguousarray(Hin.T))
    ctx.run_step(nmf.STEP_UPDATE_H)
    got = ctx.get_buffer(nmf.BUF_HT).T
    ref = fh.update_h(R.astype(np.float64), S.astype(np.float64), Hin, EPS)
    assert rel_h(got, ref) < TOL_ITER
    assert forward_error_ratio(got, ref, h_update_scale(R, S, Hin, ref)) < 1e-6


@pytest.mark.parametrize("K,T", [(16, 16), (16, 1), (20, 3), (37, 16), (48, 8)])
def test_update_w_matches_alg1(nmf, K, T):
    prob = synth.planted_dense(900, 300, 6, 41)
    W0, H0 = synth.init_factors(42 + K, 900, 300, K)
    W, H = _oracle_start(W0, H0)
    A = prob.A.astype(np.float64)
    P, Q = f32(A @ H.T), f32(H @ H.T)
    Win = f32(W)
    ctx = _dense_ctx(nmf, prob.A, K, W0, H0, tile_T=T)
    ctx.set_buffer(nmf.BUF_P, P)
    ctx.set_buffer(nmf.BUF_Q, Q)
    ctx.set_buffer(nmf.BUF_W, Win)
    ctx.run_step(nmf.STEP_UPDATE_W)
    got = ctx.get_buffer(nmf.BUF_W)
    ref = fh.update_w(P.astype(np.float64), Q.astype(np.float64), Win, EPS)
    assert rel_w(got, ref) < TOL_ITER
    print("W per-column max rel", colmax_rel(got, ref, 0))
    assert np.allclose(np.linalg.norm(got.astype(np.float64), axis=0), 1.0, atol=1e-5)


# --- one full iteration ---------------------------------------------------------

def _one_iteration(nmf, A_oracle, ctx, W0, H0):
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    W, H = _oracle_start(W0, H0)
    Wr, Hr = fh.iteration(A_oracle, W, H, EPS)
    return Wg, Hg, Wr, Hr


def test_one_iteration_dense_512x384_k16(nmf):
    """First iteration from the random start.  Its W update cancels terms of
    size ~1e5 (Q ~ 2e6), so rounding P, Q and W to FP32 once already moves W
    by ~5e-5 (max-norm, the oracle-computed floor d32).  FP32 sums of length L
    add rounding errors that grow like sqrt(L) times one rounding, so the
    tolerance is max(1e-5, sqrt(L) * d32) with L = 512, the longest inner
    dimension (A^T W sums over V = 512 rows)."""
    prob = synth.dense_small()
    W0, H0 = synth.init_factors(0xC1, 512, 384, 16)
    ctx = _dense_ctx(nmf, prob.A, 16, W0, H0)
    Wg, Hg, Wr, Hr = _one_iteration(nmf, prob.A, ctx, W0, H0)
    dW, dH = fp32_storage_sensitivity(prob.A, *_oracle_start(W0, H0))
    growth = math.sqrt(512)
    print("per-column: H", colmax_rel(Hg, Hr, 1), "W", colmax_rel(Wg, Wr, 0), "floor", dW, dH)
    assert rel_h(Hg, Hr) < max(TOL_ITER, growth * dH)
    assert rel_w(Wg, Wr) < max(TOL_ITER, growth * dW)


def test_one_iteration_dense_512x384_k16_from_iterate_10(nmf):
    """Same workload, one iteration from the oracle's 10th iterate (rounded to
    FP32 and given to both sides): the strict 1e-5 bound applies."""
    prob = synth.dense_small()
    W0, H0 = synth.init_factors(0xC1, 512, 384, 16)
    W10, H10, _ = fh.run(prob.A, W0, H0, 10)
    W10, H10 = f32(W10), f32(H10)
    ctx = _dense_ctx(nmf, prob.A, 16, W0, H0)
    ctx.set_factors(W10, H10)
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = fh.iteration(prob.A, W10.astype(np.float64), H10.astype(np.float64), EPS)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


def test_one_iteration_dense_wide_rank_from_iterate_30(nmf):
    """Dense products with K >= 96 take the 128 x 128 SIMT kernel (both
    A^T W and A H^T, with split K): 1000 x 900 is ragged against its tiles,
    K = 100.  One iteration from the oracle's 30th iterate (rounded to FP32
    and given to both sides), strict 1e-5.  At the 10th iterate this planted
    rank-100 input is still ill-conditioned (rounding P, Q and W to FP32 once
    moves W by ~5e-5); by the 30th that floor is ~2e-6, which the test checks
    so that the strict bound stays meaningful."""
    prob = synth.planted_dense(1000, 900, 100, 0xC6)
    W0, H0 = synth.init_factors(0xC6, 1000, 900, 100)
    W30, H30, _ = fh.run(prob.A, W0, H0, 30)
    W30, H30 = f32(W30), f32(H30)
    W, H = W30.astype(np.float64), H30.astype(np.float64)
    dW, dH = fp32_storage_sensitivity(prob.A, W, H)
    assert dW < 0.3 * TOL_ITER and dH < 0.3 * TOL_ITER
    ctx = _dense_ctx(nmf, prob.A, 100, W0, H0)
    ctx.set_factors(W30, H30)
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = fh.iteration(prob.A, W, H, EPS)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


def test_one_iteration_sparse_small_ragged(nmf):
    sp = synth.sparse_termdoc(2500, 1300, 51, mean_terms=30)
    W0, H0 = synth.init_factors(52, 2500, 1300, 21)
    ctx = _sparse_ctx(nmf, sp, 21, W0, H0, tile_T=6)
    Wg, Hg, Wr, Hr = _one_iteration(nmf, sp.A, ctx, W0, H0)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


@pytest.mark.parametrize("K", [80, 240, 400])
def test_one_iteration_sparse_k_sweep(nmf, K):
    """The ranks of the text-like K sweep other than 160 (different SpMM lane
    layouts, tile counts and update variants), on an 8000 x 4000 matrix of the
    same generator, one iteration against the FP64 oracle."""
    sp = synth.sparse_termdoc(8000, 4000, 0xC2 + K, mean_terms=100)
    W0, H0 = synth.init_factors(0xC2 + K + 1, 8000, 4000, K)
    ctx = _sparse_ctx(nmf, sp, K, W0, H0)
    Wg, Hg, Wr, Hr = _one_iteration(nmf, sp.A, ctx, W0, H0)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


def test_one_iteration_three_row_h_update(nmf):
    """10,000 documents at K = 320: two rows per lane group would need two
    waves of CTAs (a 64-row CTA takes more than half an SM's shared memory),
    so the H update runs three rows per lane group; its W update takes two
    rows per worker lane group and the Grams take the grouped upper-triangle
    kernel.  One iteration against the FP64 oracle."""
    sp = synth.sparse_termdoc(12000, 10000, 0xD3, mean_terms=60)
    W0, H0 = synth.init_factors(0xD4, 12000, 10000, 320)
    ctx = _sparse_ctx(nmf, sp, 320, W0, H0)
    Wg, Hg, Wr, Hr = _one_iteration(nmf, sp.A, ctx, W0, H0)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


@pytest.mark.parametrize("T", [4, 8, 12, 16])
def test_one_iteration_per_tile_w_width(nmf, T):
    """The per-tile W path at tile widths 4 .. 16 (the tile-size study; K = 21
    and 48 are multiples of none of them but 4 / 12 / 16 for 48), one
    iteration against the oracle."""
    for (V, D, seed, K) in [(2500, 1300, 51, 21), (6000, 3000, 61, 48)]:
        sp = synth.sparse_termdoc(V, D, seed, mean_terms=30)
        W0, H0 = synth.init_factors(seed + 1, V, D, K)
        ctx = _sparse_ctx(nmf, sp, K, W0, H0, tile_T=T, flags=nmf.FLAG_MULTI_LAUNCH_W)
        assert ctx.query()["tile_T"] == T
        Wg, Hg, Wr, Hr = _one_iteration(nmf, sp.A, ctx, W0, H0)
        assert rel_h(Hg, Hr) < TOL_ITER and rel_w(Wg, Wr) < TOL_ITER, (V, K, T)


@pytest.fixture(scope="module")
def text_full():
    return synth.text_20ng_like()


def test_one_iteration_text_full_size_k160(nmf, text_full):
    """26,214 x 11,314, ~1.1M nnz, K = 160: the launch configuration the
    benchmark times, one iteration against the full FP64 oracle."""
    W0, H0 = synth.init_factors(0xC2, 26214, 11314, 160)
    ctx = _sparse_ctx(nmf, text_full, 160, W0, H0)
    Wg, Hg, Wr, Hr = _one_iteration(nmf, text_full.A, ctx, W0, H0)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


@pytest.mark.parametrize("K", [80, 240, 320, 400])
def test_one_iteration_text_full_size_k_sweep(nmf, text_full, K):
    """The other ranks of the text-like K sweep at the full size, in the
    launch configurations the benchmark times there (rows per chain thread,
    rows per worker lane group and SpMM lane layouts all change with K),
    one iteration against the full FP64 oracle."""
    W0, H0 = synth.init_factors(0xC2 + K, 26214, 11314, K)
    ctx = _sparse_ctx(nmf, text_full, K, W0, H0)
    Wg, Hg, Wr, Hr = _one_iteration(nmf, text_full.A, ctx, W0, H0)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


# --- objective ------------------------------------------------------------------

def test_objective_after_50_iterations_dense_small(nmf):
    prob = synth.dense_small()
    W0, H0 = synth.init_factors(0xC1, 512, 384, 16)
    ctx = _dense_ctx(nmf, prob.A, 16, W0, H0)
    ctx.iterate(50)
    Wg, Hg = ctx.get_factors()
    Wr, Hr, _ = fh.run(prob.A, W0, H0, 50)
    f_gpu = ob.frob2_direct(prob.A, Wg, Hg)
    f_ref = ob.frob2_direct(prob.A, Wr, Hr)
    assert abs(f_gpu - f_ref) <= TOL_OBJ * f_ref
    assert Wg.min() > 0 and Hg.min() > 0


def test_objective_after_100_iterations_sparse_text_like(nmf):
    """Sparse text-like input (6,000 words x 3,000 documents, K = 32): 100
    iterations from the FP64 oracle's iterate 100, relative objective within
    1e-4 of the oracle's (measured 6e-11).  From a random start the run is
    chaotic at this level: the oracle itself, started from W0 nudged by one
    FP32 unit in the last place, ends 8e-4 away after 100 iterations."""
    import torch
    sp = synth.sparse_termdoc(6000, 3000, 22, mean_terms=60)
    W0, H0 = synth.init_factors(23, 6000, 3000, 32)
    Ws, Hs, _ = fh.run(sp.A, W0, H0, 100)
    Ws, Hs = f32(Ws), f32(Hs)
    Wr, Hr, _ = fh.run(sp.A, Ws, Hs, 100)
    f64 = ob.frob2_direct(sp.A, Wr, Hr)
    ctx = nmf.from_sparse(sp, 32, W0=torch.from_numpy(Ws).cuda(), H0=torch.from_numpy(Hs).cuda())
    ctx.iterate(100)
    f_gpu, _ = ctx.error()
    Wg, Hg = ctx.get_factors()
    f_direct = ob.frob2_direct(sp.A, Wg, Hg)
    assert abs(f_gpu - f_direct) <= 1e-5 * f_direct
    assert abs(f_direct - f64) <= TOL_OBJ * f64, (f_direct, f64)


def test_reported_objective_matches_direct_evaluation(nmf):
    """nmf_error (trace identity, FP64 accumulation of FP32 terms) against
    Eq. 2 evaluated by the oracle on the same factors."""
    sp = synth.sparse_termdoc(4000, 2000, 61, mean_terms=50)
    W0, H0 = synth.init_factors(62, 4000, 2000, 24)
    ctx = _sparse_ctx(nmf, sp, 24, W0, H0)
    f0, r0 = ctx.error()                                   # initial factors
    W, H = ctx.get_factors()
    fd = ob.frob2_direct(sp.A, W, H)
    assert abs(f0 - fd) <= 1e-5 * fd
    ctx.iterate(5)
    f5, r5 = ctx.error()
    W, H = ctx.get_factors()
    fd = ob.frob2_direct(sp.A, W, H)
    assert abs(f5 - fd) <= 1e-5 * fd
    assert abs(r5 - math.sqrt(fd / ob.norm2_A(sp.A))) <= 1e-5
    hist = ctx.history(5)
    assert abs(hist[-1] - f5) <= 1e-12 * f5
    assert np.all(np.diff(hist) <= 1e-5 * hist[0])        # non-increasing up to FP32 noise


# --- behaviour -------------------------------------------------------------------

def test_bitwise_deterministic_and_resumable(nmf):
    sp = synth.sparse_termdoc(3000, 1500, 71, mean_terms=40)
    W0, H0 = synth.init_factors(72, 3000, 1500, 32)
    a = _sparse_ctx(nmf, sp, 32, W0, H0)
    b = _sparse_ctx(nmf, sp, 32, W0, H0)
    a.iterate(5)
    b.iterate(3)
    Wb, Hb = b.get_factors()
    c = _sparse_ctx(nmf, sp, 32, W0, H0)
    c.set_factors(Wb, Hb)                                   # checkpoint -> resume
    c.iterate(2)
    Wa, Ha = a.get_factors()
    Wc, Hc = c.get_factors()
    assert np.array_equal(Wa, Wc) and np.array_equal(Ha, Hc)


def test_k1_is_clamped_power_iteration(nmf):
    prob = synth.planted_dense(200, 150, 3, 81)
    W0, H0 = synth.init_factors(82, 200, 150, 1)
    ctx = _dense_ctx(nmf, prob.A, 1, W0, H0)
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    A = prob.A.astype(np.float64)
    w = W0[:, 0].astype(np.float64)
    w /= np.linalg.norm(w)
    h1 = np.maximum(EPS, A.T @ w)
    g = np.maximum(EPS, A @ h1)
    assert np.max(np.abs(Hg[0] - h1)) <= 1e-5 * h1.max()
    assert np.max(np.abs(Wg[:, 0] - g / np.linalg.norm(g))) <= 1e-5


def test_invalid_inputs_rejected(nmf):
    import torch
    A = synth.planted_dense(50, 40, 3, 91).A.copy()
    A[3, 4] = -1.0
    with pytest.raises(nmf.NmfError) as e:
        nmf.from_dense(A, 4)
    assert e.value.status == nmf.NMF_EINVAL
    A[3, 4] = np.nan
    with pytest.raises(nmf.NmfError):
        nmf.from_dense(A, 4)
    sp = synth.sparse_termdoc(200, 100, 92, mean_terms=10)
    bad = sp.A.col_idx.copy()
    bad[5] = 100                                            # out of range
    with pytest.raises(nmf.NmfError):
        nmf.Nmf(200, 100, 4, row_ptr=torch.from_numpy(sp.A.row_ptr).cuda(),
                col_idx=torch.from_numpy(bad).cuda(), val=torch.from_numpy(sp.A.val).cuda())
    rp = sp.A.row_ptr.copy()
    rp[10], rp[11] = rp[11], rp[10] - 1                     # not monotone
    with pytest.raises(nmf.NmfError):
        nmf.Nmf(200, 100, 4, row_ptr=torch.from_numpy(rp).cuda(),
                col_idx=torch.from_numpy(sp.A.col_idx).cuda(), val=torch.from_numpy(sp.A.val).cuda())



@pytest.mark.parametrize("K", [64, 80, 160, 37])
def test_gram_partials_of_the_w_update_match_the_gram_kernel(nmf, K):
    """Within an iteration the two-grid W update's worker CTAs form the
    chunk partials of S = W^T W of the new W while the column chain runs, and
    the Gram kernel after it only reduces them.  Those partials follow the
    Gram kernel's own order for the same row chunks, so S is bit-identical to
    the Gram of the same W formed on its own (STEP_S), and within FP32
    rounding of the FP64 Gram.  K = 37 takes the ordinary Gram path (the
    chunked Gram kernel needs K >= 64)."""
    import torch
    sp = synth.sparse_termdoc(9000, 2500, 81 + K, mean_terms=50)
    W0, H0 = synth.init_factors(82 + K, 9000, 2500, K)
    ctx = nmf.from_sparse(sp, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())
    ctx.iterate(2)
    S_iter = ctx.get_buffer(nmf.BUF_S)
    ctx.run_step(nmf.STEP_S)
    S_own = ctx.get_buffer(nmf.BUF_S)
    assert np.array_equal(S_iter, S_own)
    W, _ = ctx.get_factors()
    S64 = W.astype(np.float64).T @ W.astype(np.float64)
    assert np.max(np.abs(S_iter - S64)) <= 1e-6 * np.max(np.abs(S64))

@pytest.mark.parametrize("K", [16, 37, 160])
def test_w_update_persistent_and_multi_launch_agree_with_alg1(nmf, K):
    """The two-grid (chain cluster + base workers) and the per-tile W
    updates both match Alg. 1 on a ragged K."""
    V = 3000 if K < 100 else 9000
    prob = synth.planted_dense(V, 400, 8, 101 + K)
    W0, H0 = synth.init_factors(102 + K, V, 400, K)
    W, H = _oracle_start(W0, H0)
    A = prob.A.astype(np.float64)
    P, Q = f32(A @ H.T), f32(H @ H.T)
    Win = f32(W)
    ref = fh.update_w(P.astype(np.float64), Q.astype(np.float64), Win, EPS)
    outs = []
    for flags in (0, nmf.FLAG_MULTI_LAUNCH_W):
        ctx = _dense_ctx(nmf, prob.A, K, W0, H0, flags=flags)
        ctx.set_buffer(nmf.BUF_P, P)
        ctx.set_buffer(nmf.BUF_Q, Q)
        ctx.set_buffer(nmf.BUF_W, Win)
        ctx.run_step(nmf.STEP_UPDATE_W)
        got = ctx.get_buffer(nmf.BUF_W)
        assert rel_w(got, ref) < TOL_ITER, flags
        outs.append(got)
    assert rel_w(outs[0], outs[1]) < TOL_ITER
