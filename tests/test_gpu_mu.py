"""Multiplicative updates on the GPU (`nmf_iterate_mu`, the comparator of
the paper's Sec. 2) against the FP64 MU oracle (`oracle/mu.py`): one
iteration (strict 1e-5: the rules multiply by ratios of sums of
non-negative terms, no cancellation), and 20 iterations (objective
non-increasing, within 1e-4 of the oracle's)."""

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle import mu as omu
from oracle import objective as ob
from paper_1904_07935_b300 import synth

from ._parity import rel_h, rel_w

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


def _ctx(nmf, prob, K, W0, H0):
    import torch
    kw = dict(W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())
    if hasattr(prob.A, "n_rows"):
        return nmf.from_sparse(prob, K, **kw)
    return nmf.from_dense(prob.A, K, **kw)


@pytest.mark.parametrize("case", ["dense", "sparse", "wide"])
def test_mu_one_iteration(nmf, case):
    if case == "dense":
        prob, K = synth.dense_small(), 16
    elif case == "sparse":
        prob, K = synth.sparse_termdoc(2500, 1300, 51, mean_terms=30), 21
    else:
        prob, K = synth.planted_dense(1000, 900, 100, 0xC6), 100       # 128 x 128 products
    V, D = (prob.A.n_rows, prob.A.n_cols) if hasattr(prob.A, "n_rows") else prob.A.shape
    W0, H0 = synth.init_factors(0xA1, V, D, K)
    ctx = _ctx(nmf, prob, K, W0, H0)
    ctx.iterate_mu(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = omu.iteration(prob.A, fh.normalize_init(W0), H0.astype(np.float64))
    assert rel_h(Hg, Hr) < TOL and rel_w(Wg, Wr) < TOL


def test_mu_twenty_iterations_monotone(nmf):
    sp = synth.sparse_termdoc(4000, 2000, 81, mean_terms=50)
    W0, H0 = synth.init_factors(82, 4000, 2000, 24)
    ctx = _ctx(nmf, sp, 24, W0, H0)
    fs = []
    for _ in range(20):
        ctx.iterate_mu(1)
        fs.append(ctx.error()[0])
    assert all(b <= a * (1 + 1e-6) for a, b in zip(fs, fs[1:]))
    Wr, Hr = omu.run(sp.A, W0, H0, 20)
    fr = ob.frob2_direct(sp.A, Wr, Hr)
    assert abs(fs[-1] - fr) <= 1e-4 * fr
    assert ctx.query()["launches_per_iter"] > 0          # the MU graph's own count
    prof = ctx.iterate_mu(1, profile=True)
    assert all(v > 0 for v in prof.values())
