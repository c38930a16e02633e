"""nmf_iterate_host: one iteration on caller-held factors, with the copies
captured into the iteration's graph (pinned or device buffers) or done
before and after it (pageable memory).  It adds no arithmetic: the factors
and the objective must equal those of nmf_set_factors, nmf_iterate(1),
nmf_error and nmf_get_factors on the same context configuration, bit for bit
(the same kernels in the same order; only the copies move), step after step,
with in-place buffers, after a change of buffers (a new graph), mixed with
nmf_iterate, and in the BF16 form."""

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


def _pinned(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    return t


def _reference_steps(ctx, W, H, n):
    """n round trips through the separate calls; returns the factors and
    objectives after each."""
    out = []
    W = np.ascontiguousarray(W, dtype=np.float32)
    H = np.ascontiguousarray(H, dtype=np.float32)
    for _ in range(n):
        ctx.set_factors(W, H)
        ctx.iterate(1)
        f, _ = ctx.error()
        W, H = ctx.get_factors()
        out.append((W.copy(), H.copy(), f))
    return out


def _sparse_case(nmf, K=48, flags=0):
    import torch
    sp = synth.sparse_termdoc(5000, 2200, 71, mean_terms=40)
    W0, H0 = synth.init_factors(72, 5000, 2200, K)
    mk = lambda: nmf.from_sparse(sp, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(),
                                 flags=flags)
    return mk, W0, H0


@pytest.mark.parametrize("K", [48, 37, 160])
def test_pinned_round_trips_match_separate_calls(nmf, K):
    mk, W0, H0 = _sparse_case(nmf, K)
    ref = _reference_steps(mk(), W0, H0, 3)
    ctx = mk()
    Wb, Hb = _pinned(W0), _pinned(H0)
    for W, H, f in ref:
        got = ctx.iterate_host(Wb, Hb, Wb, Hb)          # in place
        assert np.array_equal(Wb.numpy(), W) and np.array_equal(Hb.numpy(), H)
        assert got == f


def test_pageable_buffers_and_changed_pointers(nmf):
    mk, W0, H0 = _sparse_case(nmf)
    ref = _reference_steps(mk(), W0, H0, 2)
    ctx = mk()
    # pageable numpy buffers: copies before and after the iteration
    Wo = np.empty_like(W0, dtype=np.float32)
    Ho = np.empty_like(H0, dtype=np.float32)
    f = ctx.iterate_host(np.ascontiguousarray(W0, dtype=np.float32), np.ascontiguousarray(H0, dtype=np.float32),
                         Wo, Ho)
    assert np.array_equal(Wo, ref[0][0]) and np.array_equal(Ho, ref[0][1]) and f == ref[0][2]
    # pinned buffers, then other pinned buffers (the graph is captured again)
    A1, B1 = _pinned(Wo), _pinned(Ho)
    A2, B2 = _pinned(np.zeros_like(Wo)), _pinned(np.zeros_like(Ho))
    f = ctx.iterate_host(A1, B1, A2, B2)
    assert np.array_equal(A2.numpy(), ref[1][0]) and np.array_equal(B2.numpy(), ref[1][1]) and f == ref[1][2]


def test_mixed_with_device_iterations_and_null_pointers(nmf):
    """iterate_host leaves R of the new W unformed; a following nmf_iterate
    forms it.  W_in = NULL keeps the device W; outputs may be NULL."""
    mk, W0, H0 = _sparse_case(nmf)
    ref_ctx = mk()
    ref_ctx.set_factors(W0, H0)
    ref_ctx.iterate(3)
    Wr, Hr = ref_ctx.get_factors()
    fr, _ = ref_ctx.error()
    ctx = mk()
    Wb, Hb = _pinned(W0), _pinned(H0)
    ctx.iterate_host(Wb, Hb, None, None)
    ctx.iterate(1)
    f = ctx.iterate_host(None, None, Wb, Hb)
    assert np.array_equal(Wb.numpy(), Wr) and np.array_equal(Hb.numpy(), Hr) and f == fr


def test_device_buffers_dense_bf16_form(nmf):
    import torch
    prob = synth.planted_dense(1024, 768, 8, 0x5A)
    K = 32
    W0, H0 = synth.init_factors(0x5B, 1024, 768, K)
    mk = lambda: nmf.from_dense(prob.A, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(),
                                prec=nmf.PREC_BF16)
    ref = _reference_steps(mk(), W0, H0, 2)
    ctx = mk()
    Wd = torch.from_numpy(np.ascontiguousarray(W0, dtype=np.float32)).cuda()
    Hd = torch.from_numpy(np.ascontiguousarray(H0, dtype=np.float32)).cuda()
    for W, H, f in ref:
        got = ctx.iterate_host(Wd, Hd, Wd, Hd)
        torch.cuda.synchronize()
        assert np.array_equal(Wd.cpu().numpy(), W) and np.array_equal(Hd.cpu().numpy(), H)
        assert got == f
