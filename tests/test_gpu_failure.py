"""Failure path of the W update's device-side waits, without a GPU fault.

The two-grid W update replaces the paper's two host synchronisations per
column (Alg. 3) with hand-offs through global memory between the column chain
and the CTAs that form the tile bases (Alg. 2, Eqs. 4 and 6).  Every such wait
is bounded.  Here the base-forming CTAs are told to wait for one more chain
arrival than will ever come, with a 2 ms limit: their waits run out, the
status word reports the timeout once (NMF_ETIMEOUT), the chain computes the
bases those CTAs left with the same arithmetic, and the context stays usable.
Nothing traps, faults or hangs: the waits are short and bounded.

The other schedule the protocol must survive is the one a launch-serialising
tool imposes: the worker grid started only after the chain grid has finished.
The chain then forms every tile base itself, and the update must come out
bit-identical.
"""

import numpy as np
import pytest

from paper_1904_07935_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


def _ctx(nmf, sp, K, W0, H0):
    import torch
    return nmf.from_sparse(sp, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())


@pytest.mark.parametrize("K", [64, 160])
def test_w_wait_runs_out_reports_timeout_and_keeps_the_factors(nmf, K):
    sp = synth.sparse_termdoc(6000, 2500, 41, mean_terms=60)
    W0, H0 = synth.init_factors(42, 6000, 2500, K)
    ref = _ctx(nmf, sp, K, W0, H0)
    ref.iterate(1)
    W1, H1 = ref.get_factors()
    ref.iterate(1)
    W2, H2 = ref.get_factors()

    ctx = _ctx(nmf, sp, K, W0, H0)
    ctx.set_wait_limits(wait_ns=2_000_000, extra_arrivals=1)
    ctx.iterate(1)
    with pytest.raises(nmf.NmfError) as e:
        ctx.error()
    assert e.value.status == nmf.NMF_ETIMEOUT
    # Reported once; the chain formed the bases the workers gave up, with the
    # workers' arithmetic, so the factors are those of the normal update.
    W, H = ctx.get_factors()
    assert np.array_equal(W, W1) and np.array_equal(H, H1)
    # Back to the default limits: the next iteration runs clean.
    ctx.set_wait_limits(0, 0)
    ctx.iterate(1)
    ctx.error()
    W, H = ctx.get_factors()
    assert np.array_equal(W, W2) and np.array_equal(H, H2)


def test_short_wait_limit_alone_does_not_time_out(nmf):
    """A 2 ms limit is far above any wait of a normal update (microseconds)."""
    K = 96
    sp = synth.sparse_termdoc(5000, 2000, 43, mean_terms=60)
    W0, H0 = synth.init_factors(44, 5000, 2000, K)
    ref = _ctx(nmf, sp, K, W0, H0)
    ref.iterate(3)
    Wr, Hr = ref.get_factors()
    ctx = _ctx(nmf, sp, K, W0, H0)
    ctx.set_wait_limits(wait_ns=2_000_000, extra_arrivals=0)
    ctx.iterate(3)
    ctx.error()
    W, H = ctx.get_factors()
    assert np.array_equal(W, Wr) and np.array_equal(H, Hr)


def test_wait_limits_rejects_bad_arguments(nmf):
    sp = synth.sparse_termdoc(3000, 1200, 45, mean_terms=40)
    W0, H0 = synth.init_factors(46, 3000, 1200, 32)
    ctx = _ctx(nmf, sp, 32, W0, H0)
    with pytest.raises(nmf.NmfError) as e:
        ctx.set_wait_limits(wait_ns=-1)
    assert e.value.status == nmf.NMF_EINVAL
    multi = nmf.from_sparse(sp, 32, flags=nmf.FLAG_MULTI_LAUNCH_W)
    with pytest.raises(nmf.NmfError) as e:
        multi.set_wait_limits(wait_ns=1000)
    assert e.value.status == nmf.NMF_EUNSUPPORTED


@pytest.mark.parametrize("V,D,K,terms", [(1500, 900, 24, 30), (6000, 2500, 160, 60), (26214, 11314, 160, 100)])
def test_workers_after_chain_give_the_same_update(nmf, V, D, K, terms):
    """The worker grid started only after the chain grid has finished, as a
    tool that serialises launches runs the two: every worker is absent while
    the chain runs, so after each tile's hand-off window the chain claims and
    forms every tile base itself, with the workers' arithmetic in their
    order; the workers then find every base formed and only form the Gram
    partials of the new W.  Factors and objective bit-identical, no timeout."""
    sp = synth.sparse_termdoc(V, D, 47, mean_terms=terms)
    W0, H0 = synth.init_factors(48, V, D, K)
    ref = _ctx(nmf, sp, K, W0, H0)
    ref.iterate(2)
    f_ref, _ = ref.error()
    Wr, Hr = ref.get_factors()
    ctx = _ctx(nmf, sp, K, W0, H0)
    ctx.set_w_workers_after_chain(True)
    ctx.iterate(2)
    f, _ = ctx.error()
    W, H = ctx.get_factors()
    assert np.array_equal(W, Wr) and np.array_equal(H, Hr)
    assert f == f_ref
    # And back: the programmatic-dependent schedule again.
    ctx.set_w_workers_after_chain(False)
    ref.iterate(1)
    ctx.iterate(1)
    ctx.error()
    assert np.array_equal(ctx.get_factors()[0], ref.get_factors()[0])


def test_workers_after_chain_rejects_bad_arguments(nmf):
    sp = synth.sparse_termdoc(3000, 1200, 49, mean_terms=40)
    ctx = nmf.from_sparse(sp, 32)
    assert nmf.lib.nmf_set_w_workers_after_chain(ctx.h, 2) == nmf.NMF_EINVAL
    multi = nmf.from_sparse(sp, 32, flags=nmf.FLAG_MULTI_LAUNCH_W)
    with pytest.raises(nmf.NmfError) as e:
        multi.set_w_workers_after_chain(True)
    assert e.value.status == nmf.NMF_EUNSUPPORTED
