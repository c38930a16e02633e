"""Factor updates with the off-tile sums on the tensor cores
(NMF_FLAG_TC_UPDATES): the products of Eqs. 4 and 6 as TF32 pairs (3xTF32)
on tcgen05, per-plane partial sums folded with compensation, the in-tile
chains on the CUDA cores; in the H update and in the W update's tile bases.

Against Alg. 1's loops (FP64 oracle) on the same FP32 inputs: max-norm
relative difference within the FP32 path's 1e-5 up to K = 256, and the
elementwise H error within 4e-6 of the magnitude of the terms each entry is
formed from (about 2^-21 per product plus the FP32 roundings, against 1e-6
for the SIMT kernel's exact products).  At K >= 400 the tensor cores' FP32
accumulation over each 32-column plane leaves the W update at 1.2e-5
(measured; the SIMT path 4.4e-6), held to 2e-5 there.  Shapes are ragged
against the 128-row CTAs, the 32-column planes and the 16-column tiles, up
to K = 512."""

import numpy as np
import pytest

from oracle import fast_hals as fh
from paper_1904_07935_b300 import synth

from ._parity import f32, forward_error_ratio, h_update_scale, rel_h, rel_w

pytestmark = pytest.mark.gpu

EPS = 1e-16
TOL_ITER = 1e-5


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


@pytest.mark.parametrize("K,D", [(16, 700), (37, 700), (48, 1000), (160, 700), (250, 300), (512, 600)])
def test_update_h_tc_matches_alg1(nmf, K, D):
    V = max(260, K + 8)
    prob = synth.planted_dense(V, D, 6, 31)
    W0, H0 = synth.init_factors(32 + K, V, D, K)
    W, H = fh.normalize_init(W0), H0.astype(np.float64)
    A = prob.A.astype(np.float64)
    R, S = f32(A.T @ W), f32(W.T @ W)
    Hin = f32(H)
    ref = fh.update_h(R.astype(np.float64), S.astype(np.float64), Hin, EPS)
    out = {}
    for flags in (0, nmf.FLAG_TC_UPDATES):
        ctx = _dense_ctx(nmf, prob.A, K, W0, H0, flags=flags)
        ctx.set_buffer(nmf.BUF_R, R)
        ctx.set_buffer(nmf.BUF_S, S)
        ctx.set_buffer(nmf.BUF_HT, np.ascontiguousarray(Hin.T))
        ctx.run_step(nmf.STEP_UPDATE_H)
        out[flags] = ctx.get_buffer(nmf.BUF_HT).T
    got = out[nmf.FLAG_TC_UPDATES]
    fe = forward_error_ratio(got, ref, h_update_scale(R, S, Hin, ref))
    print(f"K={K} D={D}: rel {rel_h(got, ref):.3e} (simt {rel_h(out[0], ref):.3e}) fwd {fe:.3e}")
    assert rel_h(got, ref) < TOL_ITER
    assert fe < 4e-6


@pytest.mark.parametrize("K", [32, 160])
def test_one_iteration_sparse_tc_updates(nmf, K):
    import torch
    sp = synth.sparse_termdoc(6000, 2700, 61, mean_terms=60)
    W0, H0 = synth.init_factors(62, 6000, 2700, K)
    ctx = nmf.from_sparse(sp, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(),
                          flags=nmf.FLAG_TC_UPDATES)
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = fh.iteration(sp.A, fh.normalize_init(W0), H0.astype(np.float64), EPS)
    print(f"sparse K={K}: W {rel_w(Wg, Wr):.3e} H {rel_h(Hg, Hr):.3e}")
    assert rel_h(Hg, Hr) < TOL_ITER and rel_w(Wg, Wr) < TOL_ITER


def test_dense_from_iterate_10_tc_updates(nmf):
    """The planted 512 x 384 input from the oracle's 10th iterate (where the
    FP32 storage floor is below the tolerance)."""
    import torch
    prob = synth.dense_small()
    W0, H0 = synth.init_factors(0xC1, 512, 384, 16)
    W10, H10, _ = fh.run(prob.A, W0, H0, 10)
    W10, H10 = f32(W10), f32(H10)
    ctx = _dense_ctx(nmf, prob.A, 16, W10, H10, flags=nmf.FLAG_TC_UPDATES)
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = fh.iteration(prob.A, fh.normalize_init(W10), H10.astype(np.float64), EPS)
    print(f"dense 512x384 from it 10: W {rel_w(Wg, Wr):.3e} H {rel_h(Hg, Hr):.3e}")
    assert rel_h(Hg, Hr) < TOL_ITER and rel_w(Wg, Wr) < TOL_ITER


@pytest.mark.parametrize("K,V", [(16, 3000), (37, 3000), (160, 9000), (400, 9000)])
def test_update_w_tc_matches_alg1(nmf, K, V):
    """The W update with the tile bases formed on the tensor cores by the
    worker clusters (the column chain unchanged) against Alg. 1's W loop."""
    D = max(400, K + 16)
    prob = synth.planted_dense(V, D, 8, 101 + K)
    W0, H0 = synth.init_factors(102 + K, V, D, K)
    W, H = fh.normalize_init(W0), H0.astype(np.float64)
    A = prob.A.astype(np.float64)
    P, Q = f32(A @ H.T), f32(H @ H.T)
    Win = f32(W)
    ref = fh.update_w(P.astype(np.float64), Q.astype(np.float64), Win, EPS)
    out = {}
    for flags in (0, nmf.FLAG_TC_UPDATES):
        ctx = _dense_ctx(nmf, prob.A, K, W0, H0, flags=flags)
        ctx.set_buffer(nmf.BUF_P, P)
        ctx.set_buffer(nmf.BUF_Q, Q)
        ctx.set_buffer(nmf.BUF_W, Win)
        ctx.run_step(nmf.STEP_UPDATE_W)
        out[flags] = ctx.get_buffer(nmf.BUF_W)
    got = out[nmf.FLAG_TC_UPDATES]
    print(f"W K={K} V={V}: rel {rel_w(got, ref):.3e} (simt {rel_w(out[0], ref):.3e})")
    assert rel_w(got, ref) < (TOL_ITER if K <= 256 else 2e-5)
