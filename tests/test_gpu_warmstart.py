"""Learned warm start (fixed-W H subproblem) on the GPU against the oracle.

* Network forward / backward: the tensor-core products take BF16 operands
  with FP32 accumulation, so the GPU is compared with the oracle network in
  its reduced-precision-product form (operands of every product rounded to
  BF16, FP64 otherwise) within 2e-3 normwise (FP32 accumulation plus rare
  BF16 rounding flips of FP32-vs-FP64 intermediates), and with the plain
  FP64 network within 2e-2 (the BF16 operand error).
* Adam: given the GPU's own gradients, the update matches the oracle's
  adam_step to FP32 rounding.
* Sweeps: nmf_warm_h repeats the H loop of Alg. 1 with S = W^T W fixed; a
  few sweeps match the oracle's update_h sweeps (same cold start, the
  SplitMix draws nmf_init uses for H) within 2e-5 max-norm relative, and
  run to convergence they reach the oracle's fixed-W optimum h*.
"""

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle import mlp as om
from oracle import nnls
from oracle.bf16 import round_bf16
from paper_1904_07935_b300 import synth

from ._parity import rel_h

pytestmark = pytest.mark.gpu

EPS = 1e-16
V, D, K = 3000, 1500, 32
HID = 64


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


@pytest.fixture(scope="module")
def fixed(nmf):
    """A context whose W is the 20th iterate of a small text-like problem."""
    sp = synth.sparse_termdoc(V, D, 1701, mean_terms=30)
    ctx = nmf.from_sparse(sp, K, seed=1702)
    ctx.iterate(20)
    W = ctx.get_factors()[0].astype(np.float64)
    return ctx, W


def _docs(n, seed):
    return synth.sparse_termdoc(V, n, seed, mean_terms=30)


def _params(seed, K=K, H=HID):
    rng = np.random.default_rng(seed)
    out = []
    for i, o in [(K, H), (H, H), (H, K)]:
        out += [rng.normal(scale=1.0 / np.sqrt(i), size=(i, o)).astype(np.float32),
                rng.normal(scale=0.1, size=o).astype(np.float32)]
    return out


def _nrel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


# --- network ---------------------------------------------------------------

def test_mlp_forward_against_oracle(nmf):
    import torch
    m = nmf.Mlp(K, HID, seed=5)
    p = _params(11)
    m.set_params(p)
    rng = np.random.default_rng(12)
    X = np.abs(rng.normal(size=(300, K))).astype(np.float32)            # 300 rows: ragged vs 128-row tiles
    Y = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    yb, _ = om.forward(p, X, operand_round=round_bf16)
    y64, _ = om.forward(p, X)
    assert _nrel(Y, yb) < 2e-3
    assert _nrel(Y, y64) < 2e-2


def test_mlp_gradients_against_oracle(nmf):
    import torch
    m = nmf.Mlp(K, HID, seed=5)
    p = _params(21)
    m.set_params(p)
    rng = np.random.default_rng(22)
    X = np.abs(rng.normal(size=(203, K))).astype(np.float32)
    T = np.abs(rng.normal(size=(203, K))).astype(np.float32)
    g, loss = m.grads(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    yb, cb = om.forward(p, X, operand_round=round_bf16)
    gb = om.backward(p, cb, yb, T, operand_round=round_bf16)
    y64, c64 = om.forward(p, X)
    g64 = om.backward(p, c64, y64, T)
    for a, b, c in zip(g, gb, g64):
        assert _nrel(a, b) < 2e-3
        assert _nrel(a, c) < 2e-2
    assert abs(loss - np.mean((yb - T) ** 2)) <= 2e-3 * np.mean((yb - T) ** 2)


def test_adam_steps_against_oracle(nmf):
    import torch
    m = nmf.Mlp(K, HID, seed=5)
    p0 = _params(31)
    m.set_params(p0)
    rng = np.random.default_rng(32)
    X = torch.from_numpy(np.abs(rng.normal(size=(128, K))).astype(np.float32)).cuda()
    T = torch.from_numpy(np.abs(rng.normal(size=(128, K))).astype(np.float32)).cuda()
    lr = 1e-2
    zeros = [np.zeros(a.shape) for a in p0]
    g1, _ = m.grads(X, T)
    m.train_step(X, T, lr=lr)
    p1 = m.get_params()
    o1, m1, v1 = om.adam_step([a.astype(np.float64) for a in p0], [a.astype(np.float64) for a in g1], zeros, zeros,
                              1, lr=lr)
    for a, b in zip(p1, o1):
        assert np.max(np.abs(a - b)) <= 1e-6 * lr + 2e-7 * np.max(np.abs(b))
    g2, _ = m.grads(X, T)
    m.train_step(X, T, lr=lr)
    p2 = m.get_params()
    o2, _, _ = om.adam_step([a.astype(np.float64) for a in p1], [a.astype(np.float64) for a in g2], m1, v1, 2, lr=lr)
    for a, b in zip(p2, o2):
        assert np.max(np.abs(a - b)) <= 1e-5 * lr + 2e-7 * np.max(np.abs(b))


def test_mlp_rejects_bad_sizes(nmf):
    with pytest.raises(nmf.NmfError):
        nmf.Mlp(K, 60)                       # hidden not a multiple of 8
    with pytest.raises(nmf.NmfError):
        nmf.Mlp(0, 64)


# --- fixed-W sweeps --------------------------------------------------------

def test_sweeps_against_oracle(nmf, fixed):
    ctx, W = fixed
    docs = _docs(700, 1711)
    out = nmf.warm_h(ctx, docs, tol=0.0, max_sweeps=3, want_R=True, seed=77)
    assert out["sweeps"] == 3
    R = np.asarray(docs.A.to_scipy().T @ W)
    S = W.T @ W
    assert np.max(np.abs(out["R"] - R)) <= 1e-6 * np.max(np.abs(R))
    H = synth.init_factors(77, V, 700, K)[1].astype(np.float64)        # the cold start nmf_init draws
    for _ in range(3):
        H = fh.update_h(R, S, H, EPS)
    assert rel_h(out["H"], H) < 2e-5


def test_sweeps_reach_the_fixed_w_optimum(nmf, fixed):
    ctx, W = fixed
    docs = _docs(400, 1721)
    R = np.asarray(docs.A.to_scipy().T @ W)
    S = W.T @ W
    H0 = synth.init_factors(78, V, 400, K)[1].astype(np.float64)
    Hs, _ = nnls.hals_sweeps(R, S, H0, EPS, tol=1e-12, max_sweeps=20000)
    out = nmf.warm_h(ctx, docs, tol=1e-4, max_sweeps=3000, H_ref=Hs.astype(np.float32), seed=78)
    assert out["sweeps"] < 3000
    assert out["trace"][-1] <= 1e-4
    assert np.linalg.norm(out["H"] - Hs) / np.linalg.norm(Hs) <= 1.01e-4


def test_warm_start_begins_at_the_network_output(nmf, fixed):
    import torch
    ctx, W = fixed
    docs = _docs(300, 1731)
    m = nmf.Mlp(K, HID, seed=9)
    out = nmf.warm_h(ctx, docs, mlp=m, tol=0.0, max_sweeps=0, want_R=True)
    assert out["sweeps"] == 0
    Y = m.forward(torch.from_numpy(out["R"]).cuda()).cpu().numpy()
    assert np.array_equal(out["H"], Y.T)


def test_trained_network_needs_fewer_sweeps(nmf, fixed):
    import torch
    ctx, W = fixed
    S = W.T @ W
    train, evald = _docs(3000, 1741), _docs(600, 1742)
    tr = nmf.warm_h(ctx, train, tol=1e-7, max_sweeps=3000, want_R=True, seed=1)
    Rt = torch.from_numpy(tr["R"]).cuda()
    Ht = torch.from_numpy(np.ascontiguousarray(tr["H"].T)).cuda()
    m = nmf.Mlp(K, HID, seed=10)
    for ep in range(60):
        perm = torch.randperm(Rt.shape[0], generator=torch.Generator().manual_seed(ep)).cuda()
        for i in range(0, Rt.shape[0], 256):
            idx = perm[i:i + 256]
            m.train_step(Rt[idx].contiguous(), Ht[idx].contiguous(), lr=2e-3)
    Re = np.asarray(evald.A.to_scipy().T @ W)
    H0 = synth.init_factors(2, V, 600, K)[1].astype(np.float64)
    Hs, _ = nnls.hals_sweeps(Re, S, H0, EPS, tol=1e-12, max_sweeps=20000)
    Hs32 = Hs.astype(np.float32)
    cold = nmf.warm_h(ctx, evald, tol=1e-3, max_sweeps=3000, H_ref=Hs32, seed=2)
    warm = nmf.warm_h(ctx, evald, mlp=m, tol=1e-3, max_sweeps=3000, H_ref=Hs32)
    print("sweeps to 1e-3: cold", cold["sweeps"], "warm", warm["sweeps"])
    assert warm["trace"][-1] <= 1e-3 and cold["trace"][-1] <= 1e-3
    assert warm["sweeps"] < cold["sweeps"]


def test_warm_h_rejects_mismatches(nmf, fixed):
    ctx, _ = fixed
    other = synth.sparse_termdoc(V + 5, 50, 1751, mean_terms=10)
    with pytest.raises(nmf.NmfError) as e:
        nmf.warm_h(ctx, other, max_sweeps=1)
    assert e.value.status == nmf.NMF_EINVAL
    m = nmf.Mlp(K + 8, HID)
    with pytest.raises(nmf.NmfError):
        nmf.warm_h(ctx, _docs(20, 1752), mlp=m, max_sweeps=1)


@pytest.mark.parametrize("Kw", [48, 32])
def test_sweep_checks_on_the_device(nmf, Kw):
    """The stopping values formed on the device (in the H update's write-back
    for K > 32, by a pass of their own for the row-per-warp form) equal the
    relative changes of the returned iterates, and a loop that meets tol in
    its second chunk of 32 sweeps returns exactly the H of that sweep (the
    later sweeps of the chunk leave it unchanged)."""
    sp = synth.sparse_termdoc(V, D, 1731, mean_terms=30)
    ctx = nmf.from_sparse(sp, Kw, seed=1732)
    ctx.iterate(10)
    docs = _docs(600, 1733)
    Hs = [nmf.warm_h(ctx, docs, tol=0.0, max_sweeps=s, seed=79)["H"].astype(np.float64) for s in (1, 2, 3)]
    out = nmf.warm_h(ctx, docs, tol=0.0, max_sweeps=3, seed=79)
    assert np.array_equal(out["H"], Hs[2].astype(np.float32))
    for s in (1, 2):
        want = np.linalg.norm(Hs[s] - Hs[s - 1]) / np.linalg.norm(Hs[s - 1])
        assert abs(out["trace"][s] - want) <= 1e-5 * want
    ref = Hs[2].astype(np.float32)
    out_r = nmf.warm_h(ctx, docs, tol=0.0, max_sweeps=2, H_ref=ref, seed=79)
    for s in (0, 1):
        want = np.linalg.norm(Hs[s] - Hs[2]) / np.linalg.norm(Hs[2])
        assert abs(out_r["trace"][s] - want) <= 1e-5 * want
    # tol = the smallest change of 60 sweeps, met in the second chunk or
    # later: the loop stops at the first sweep whose change is <= tol
    long = nmf.warm_h(ctx, docs, tol=0.0, max_sweeps=60, seed=79)
    tr = long["trace"]
    t32 = np.float32(tr[32:].min())
    if float(t32) < tr[32:].min():
        t32 = np.nextafter(t32, np.float32(np.inf))       # tol is passed as a float
    tol = float(t32)
    assert np.any(tr <= tol)
    first = int(np.argmax(tr <= tol)) + 1
    stop = nmf.warm_h(ctx, docs, tol=tol, max_sweeps=60, seed=79)
    assert stop["sweeps"] == first and stop["trace"][-1] <= tol
    again = nmf.warm_h(ctx, docs, tol=0.0, max_sweeps=first, seed=79)
    assert np.array_equal(stop["H"], again["H"])
