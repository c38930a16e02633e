"""Alg. 1 as written on the GPU (`nmf_iterate_alg1`: column-by-column
updates, no tiling), the comparator of the regrouped form: one iteration
against the FP64 oracle (strict 1e-5, on cases whose FP32 storage floor is
far below it), agreement with the regrouped iteration, the step profile,
and mixing the two forms on one context."""

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle import objective as ob
from paper_1904_07935_b300 import synth

from ._parity import f32, rel_h, rel_w

pytestmark = pytest.mark.gpu

EPS = 1e-16
TOL = 1e-5


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


def _sparse(nmf, sp, K, W0, H0):
    import torch
    return nmf.from_sparse(sp, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())


def _dense(nmf, A, K, W0, H0):
    import torch
    return nmf.from_dense(A, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())


def test_alg1_one_iteration_sparse_ragged(nmf):
    sp = synth.sparse_termdoc(2500, 1300, 51, mean_terms=30)
    W0, H0 = synth.init_factors(52, 2500, 1300, 21)
    ctx = _sparse(nmf, sp, 21, W0, H0)
    ctx.iterate_alg1(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = fh.iteration(sp.A, fh.normalize_init(W0), H0.astype(np.float64), EPS)
    assert rel_h(Hg, Hr) < TOL and rel_w(Wg, Wr) < TOL


def test_alg1_one_iteration_dense_from_iterate_10(nmf):
    prob = synth.dense_small()
    W0, H0 = synth.init_factors(0xC1, 512, 384, 16)
    W10, H10, _ = fh.run(prob.A, W0, H0, 10)
    W10, H10 = f32(W10), f32(H10)
    ctx = _dense(nmf, prob.A, 16, W0, H0)
    ctx.set_factors(W10, H10)
    ctx.iterate_alg1(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = fh.iteration(prob.A, W10.astype(np.float64), H10.astype(np.float64), EPS)
    assert rel_h(Hg, Hr) < TOL and rel_w(Wg, Wr) < TOL


def test_alg1_matches_regrouped_form(nmf):
    """One iteration from the random start (K = 48: dot products of more than
    one pass of 32 lanes): the two GPU forms and the oracle agree.  (The
    second iteration of these text-like inputs is not a fair comparison:
    rounding the stored intermediates to FP32 once moves its W by 6-17%.)"""
    sp = synth.sparse_termdoc(6000, 3000, 61, mean_terms=60)
    W0, H0 = synth.init_factors(62, 6000, 3000, 48)
    a, b = _sparse(nmf, sp, 48, W0, H0), _sparse(nmf, sp, 48, W0, H0)
    a.iterate_alg1(1)
    b.iterate(1)
    Wa, Ha = a.get_factors()
    Wb, Hb = b.get_factors()
    Wr, Hr = fh.iteration(sp.A, fh.normalize_init(W0), H0.astype(np.float64), EPS)
    assert rel_w(Wa, Wr) < TOL and rel_h(Ha, Hr) < TOL
    assert rel_w(Wa, Wb) < 2 * TOL and rel_h(Ha, Hb) < 2 * TOL
    # nmf_query reports the launches of the form run last: K column launches
    # for H and 2K for W (Alg. 1 as written) against a handful for the
    # regrouped form.
    la, lb = a.query()["launches_per_iter"], b.query()["launches_per_iter"]
    assert la >= 3 * 48 and 0 < lb < 48


def test_alg1_profile_and_mixing(nmf):
    """The step profile, then the two forms interleaved on one context from
    the oracle's 2nd iterate (FP32 storage floors 2.3e-6 .. 1.5e-7 over the
    next iterations): every step, whichever form, is one Alg. 1 iteration of
    the factors it found (so each form leaves S = W^T W and R = A^T W valid
    for the other)."""
    sp = synth.sparse_termdoc(3000, 1500, 71, mean_terms=40)
    W0, H0 = synth.init_factors(72, 3000, 1500, 32)
    ctx = _sparse(nmf, sp, 32, W0, H0)
    prof = ctx.iterate_alg1(1, profile=True)
    assert set(prof) == set(ctx.PROFILE_STEPS) and all(v > 0 for v in prof.values())
    W2, H2, _ = fh.run(sp.A, W0, H0, 2)
    ctx.set_factors(f32(W2), f32(H2))
    for form in ("alg1", "tiled", "alg1"):
        Wp, Hp = ctx.get_factors()
        if form == "alg1":
            ctx.iterate_alg1(1)
        else:
            ctx.iterate(1)
        Wg, Hg = ctx.get_factors()
        Wr, Hr = fh.iteration(sp.A, Wp.astype(np.float64), Hp.astype(np.float64), EPS)
        assert rel_w(Wg, Wr) < TOL and rel_h(Hg, Hr) < TOL, form
    f, _ = ctx.error()
    assert abs(f - ob.frob2_direct(sp.A, Wg, Hg)) <= 1e-5 * f
