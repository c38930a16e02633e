"""Edge cases of the GPU path against the FP64 oracle: an all-zero A (every
factor entry ends at the clamp floor or its normalised value), a single row
or column (K = 1), the largest rank this build supports (K = 512: the widest
SpMM lane layout, 128 x 128 Gram tiles, the widest update tiles), and a
dense A with many exact zeros."""

import numpy as np
import pytest

from oracle import fast_hals as fh
from paper_1904_07935_b300 import synth

from ._parity import rel_h, rel_w

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


def _dense(nmf, A, K, W0, H0):
    import torch
    return nmf.from_dense(A, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())


def _one(nmf, ctx, A, W0, H0):
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    Wr, Hr = fh.iteration(A, fh.normalize_init(W0), H0.astype(np.float64), EPS)
    return Wg, Hg, Wr, Hr


def test_all_zero_matrix_rejected(nmf):
    """A = 0 (no non-zeros, or a dense zero matrix): the relative error
    ||A - WH|| / ||A|| is undefined, so nmf_init refuses it (NMF_EINVAL)."""
    import torch
    V, D, K = 300, 200, 8
    rp = torch.zeros(V + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    va = torch.zeros(0, dtype=torch.float32, device="cuda")
    with pytest.raises(nmf.NmfError) as e:
        nmf.Nmf(V, D, K, row_ptr=rp, col_idx=ci, val=va)
    assert e.value.status == nmf.NMF_EINVAL
    with pytest.raises(nmf.NmfError) as e:
        nmf.from_dense(np.zeros((V, D), dtype=np.float32), K)
    assert e.value.status == nmf.NMF_EINVAL


@pytest.mark.parametrize("shape", [(1, 50), (60, 1), (1, 1)])
def test_single_row_or_column(nmf, shape):
    V, D = shape
    rng = np.random.default_rng(V * 100 + D)
    A = (rng.random((V, D)) + 0.1).astype(np.float32)
    W0, H0 = synth.init_factors(7, V, D, 1)
    ctx = _dense(nmf, A, 1, W0, H0)
    Wg, Hg, Wr, Hr = _one(nmf, ctx, A, W0, H0)
    assert rel_h(Hg, Hr) < TOL and rel_w(Wg, Wr) < TOL


def test_largest_rank_sparse(nmf):
    """K = 512 (the build's maximum) on a 1600 x 900 text-like matrix."""
    import torch
    K = 512
    sp = synth.sparse_termdoc(1600, 900, 91, mean_terms=120)
    W0, H0 = synth.init_factors(92, 1600, 900, K)
    ctx = nmf.from_sparse(sp, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())
    Wg, Hg, Wr, Hr = _one(nmf, ctx, sp.A, W0, H0)
    assert rel_h(Hg, Hr) < TOL and rel_w(Wg, Wr) < TOL
    with pytest.raises(nmf.NmfError) as e:
        nmf.from_sparse(sp, 513)
    assert e.value.status == nmf.NMF_EUNSUPPORTED


def test_dense_with_many_zeros(nmf):
    rng = np.random.default_rng(11)
    A = rng.random((700, 500)).astype(np.float32)
    A[rng.random(A.shape) < 0.7] = 0.0                      # 70% exact zeros, some all-zero rows
    A[5] = 0.0
    A[:, 7] = 0.0
    W0, H0 = synth.init_factors(12, 700, 500, 24)
    ctx = _dense(nmf, A, 24, W0, H0)
    Wg, Hg, Wr, Hr = _one(nmf, ctx, A, W0, H0)
    assert rel_h(Hg, Hr) < TOL and rel_w(Wg, Wr) < TOL
