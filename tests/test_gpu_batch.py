"""Batched form: independent problems advanced together by one CUDA graph
(nmf_batch_*).  The batch adds no arithmetic, so each member must equal the
same problem run alone: bit-exact when the configuration is the same (the
kernels are deterministic), and within the one-iteration FP32 tolerance of
the FP64 oracle (Alg. 1) when the autotuner changed a member's schedule
(the chain's cluster size, the W tile width, the SpMM split lengths: each a
different but fixed order of the same sums)."""

import numpy as np
import pytest

from oracle import fast_hals as fh
from paper_1904_07935_b300 import synth

from ._parity import rel_h, rel_w

pytestmark = pytest.mark.gpu

EPS = 1e-16
TOL_ITER = 1e-5

# (V, D, mean distinct terms per document, K): ragged against 16-column tiles,
# row counts that fit clusters of 4, 8 and 16 CTAs.
SHAPES = [(1200, 700, 12, 16), (3100, 900, 25, 21), (5000, 2200, 30, 32), (9000, 1500, 40, 48),
          (16000, 3000, 60, 64)]


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


@pytest.fixture(scope="module")
def problems():
    out = []
    for i, (V, D, L, K) in enumerate(SHAPES):
        sp = synth.sparse_termdoc(V, D, 900 + i, mean_terms=L)
        W0, H0 = synth.init_factors(950 + i, V, D, K)
        out.append((sp, K, W0, H0))
    return out


def _ctx(nmf, sp, K, W0, H0, **kw):
    import torch
    return nmf.from_sparse(sp, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(), **kw)


def test_batch_equals_solo_runs_bit_exact(nmf, problems):
    solo = []
    for sp, K, W0, H0 in problems:
        c = _ctx(nmf, sp, K, W0, H0, flags=nmf.FLAG_MULTI_LAUNCH_W)
        c.iterate(3)
        solo.append(c.get_factors())
    members = [_ctx(nmf, sp, K, W0, H0) for sp, K, W0, H0 in problems]
    b = nmf.Batch(members, autotune=False)
    b.iterate(3)
    for m, (Ws, Hs) in zip(members, solo):
        W, H = m.get_factors()
        assert np.array_equal(W, Ws) and np.array_equal(H, Hs)
    b.close()


def test_batch_autotuned_one_iteration_against_oracle(nmf, problems):
    members = [_ctx(nmf, sp, K, W0, H0) for sp, K, W0, H0 in problems]
    b = nmf.Batch(members, autotune=True)
    sizes = [b.query(i)[0] for i in range(len(members))]
    assert all(s in (4, 8, 16) for s in sizes)
    segs = (128, 256, 512, 1024, 1 << 30)
    for i in range(len(members)):
        s = b.schedule(i)
        assert s["tile_T"] in (8, 12, 16) and s["spmm_seg_P"] in segs and s["spmm_seg_R"] in segs
    b.iterate(1)
    for m, (sp, K, W0, H0) in zip(members, problems):
        Wg, Hg = m.get_factors()
        Wr, Hr = fh.iteration(sp.A, fh.normalize_init(W0), H0.astype(np.float64), EPS)
        assert rel_h(Hg, Hr) < TOL_ITER
        assert rel_w(Wg, Wr) < TOL_ITER
    b.close()


def test_autotuning_does_not_advance_the_factors(nmf, problems):
    members = [_ctx(nmf, sp, K, W0, H0) for sp, K, W0, H0 in problems[:3]]
    before = [m.get_factors() for m in members]
    b = nmf.Batch(members, autotune=True)
    for m, (W0, H0) in zip(members, before):
        W, H = m.get_factors()
        assert np.array_equal(W, W0) and np.array_equal(H, H0)
    b.close()


def test_batch_then_member_calls_see_the_result(nmf, problems):
    sp, K, W0, H0 = problems[1]
    m1 = _ctx(nmf, sp, K, W0, H0)
    m2 = _ctx(nmf, *problems[2])
    b = nmf.Batch([m1, m2], autotune=False)
    b.iterate(2)
    f_b, _ = m1.error()
    solo = _ctx(nmf, sp, K, W0, H0, flags=nmf.FLAG_MULTI_LAUNCH_W)
    solo.iterate(2)
    f_s, _ = solo.error()
    assert f_b == f_s
    m1.iterate(1)            # the member's own graph is re-captured in the per-tile W form
    solo.iterate(1)
    assert np.array_equal(m1.get_factors()[0], solo.get_factors()[0])
    b.close()


def test_batch_submit(nmf, problems):
    specs = []
    for sp, K, W0, H0 in problems[:3]:
        import torch
        rp, ci, va = nmf.sparse_device(sp)
        specs.append(dict(V=sp.A.n_rows, D=sp.A.n_cols, K=K, row_ptr=rp, col_idx=ci, val=va,
                          W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda()))
    ctxs = nmf.batch_submit(specs, 1)
    for m, (sp, K, W0, H0) in zip(ctxs, problems[:3]):
        Wg, Hg = m.get_factors()
        Wr, Hr = fh.iteration(sp.A, fh.normalize_init(W0), H0.astype(np.float64), EPS)
        assert rel_h(Hg, Hr) < TOL_ITER and rel_w(Wg, Wr) < TOL_ITER


def test_batch_rejects_bad_members(nmf, problems):
    import torch
    sp, K, W0, H0 = problems[0]
    m = _ctx(nmf, sp, K, W0, H0)
    with pytest.raises(nmf.NmfError) as e:
        nmf.Batch([m, m])
    assert e.value.status == nmf.NMF_EINVAL
    with pytest.raises(nmf.NmfError):
        nmf.Batch([])
    s = torch.cuda.Stream()
    a1 = _ctx(nmf, sp, K, W0, H0, stream=s)
    a2 = _ctx(nmf, sp, K, W0, H0, stream=s)
    with pytest.raises(nmf.NmfError) as e:
        nmf.Batch([a1, a2])                   # members sharing a stream
    assert e.value.status == nmf.NMF_EINVAL
