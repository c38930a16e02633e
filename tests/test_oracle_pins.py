"""Pins for the FP64 oracle: facts fixed by the paper or by mathematics,
independent of the oracle's own formulas (CPU only)."""

import math
import os

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle import mlp, nnls, objective as ob, pl_nmf, tile_model as tm
from paper_1904_07935_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 1e-16


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        rows = [ln.split(None, 2) for ln in f if ln.strip() and not ln.startswith("#")]
    return {r[0]: float(r[1]) for r in rows}


def _dense(V, D, K0, seed):
    return synth.planted_dense(V, D, K0, seed).A.astype(np.float64)


# --- Sec. 3.3: the tiled reorder performs the same operations -----------------

@pytest.mark.parametrize("K,T", [(7, 1), (7, 2), (7, 3), (7, 5), (7, 7), (16, 16),
                                 (20, 3), (20, 16), (33, 8)])
def test_reorder_identity(K, T):
    """Alg. 2 (three phases) equals Alg. 1 (sequential k loop) to rounding,
    for T dividing K, T not dividing K, T = 1 and T = K."""
    A = _dense(45, 38, 5, 7)
    W0, H0 = synth.init_factors(21 + K, 45, 38, K)
    W = fh.normalize_init(W0)
    H = H0.astype(np.float64)
    tr = {}
    W1, H1 = fh.iteration(A, W, H, EPS, trace=tr)
    Hp = pl_nmf.update_h(tr["R"], tr["S"], H, T, EPS)
    Wp = pl_nmf.update_w(tr["P"], tr["Q"], W, T, EPS)
    assert np.max(np.abs(Hp - H1)) <= 1e-12 * np.max(np.abs(H1))
    assert np.max(np.abs(Wp - W1)) <= 1e-12 * np.max(np.abs(W1))


def test_reorder_identity_sparse_with_empty_rows():
    sp = synth.sparse_termdoc(400, 150, 3, mean_terms=15)
    assert np.any(np.diff(sp.A.row_ptr) == 0)          # Zipf tail words never drawn
    W0, H0 = synth.init_factors(4, 400, 150, 12)
    W = fh.normalize_init(W0)
    tr = {}
    W1, H1 = fh.iteration(sp.A, W, H0, EPS, trace=tr)
    for T in (4, 5):
        assert np.allclose(pl_nmf.update_w(tr["P"], tr["Q"], W, T, EPS), W1, rtol=0, atol=1e-13)
        assert np.allclose(pl_nmf.update_h(tr["R"], tr["S"], H0, T, EPS), H1, rtol=0,
                           atol=1e-12 * np.abs(H1).max())
    # an empty row of A has P = 0, so every entry is clamped to eps before the
    # column is normalised: all empty rows share the column's minimum value
    empty = np.where(np.diff(sp.A.row_ptr) == 0)[0]
    assert np.all(W1[empty] == W1[empty[0]][None, :])
    assert np.all(W1[empty[0]] == W1.min(axis=0))


# --- monotone objective --------------------------------------------------------

def test_objective_non_increasing():
    """With unit-norm W columns each coordinate step is an exact minimiser, so
    the objective never increases (up to rounding) after the first iteration."""
    A = _dense(80, 60, 6, 3)
    W0, H0 = synth.init_factors(8, 80, 60, 9)
    W, H = fh.normalize_init(W0), H0.astype(np.float64)
    fs = []
    for _ in range(60):
        W, H = fh.iteration(A, W, H, EPS)
        fs.append(ob.frob2_direct(A, W, H))
    for a, b in zip(fs, fs[1:]):
        assert b <= a * (1 + 1e-12)
    assert fs[-1] < 0.5 * fs[0]


def test_non_negativity_and_unit_columns():
    sp = synth.sparse_termdoc(300, 120, 5, mean_terms=12)
    W0, H0 = synth.init_factors(6, 300, 120, 10)
    W, H, _ = fh.run(sp.A, W0, H0, 5)
    # H is clamped at eps; W is clamped at eps and then divided by its column
    # norm, so it stays strictly positive
    assert H.min() >= EPS and W.min() > 0
    assert np.allclose(np.linalg.norm(W, axis=0), 1.0, atol=1e-14)


# --- K = 1: clamped power iteration --------------------------------------------

def test_k1_one_step_closed_form():
    """K = 1, unit w: h <- max(eps, A^T w), w <- normalise(max(eps, A h))."""
    A = _dense(40, 30, 3, 2)
    W0, H0 = synth.init_factors(3, 40, 30, 1)
    w = W0[:, 0].astype(np.float64)
    w /= math.sqrt(float(np.dot(w, w)))
    h1 = np.maximum(EPS, A.T @ w)
    g = np.maximum(EPS, A @ h1)
    w1 = g / math.sqrt(float(np.dot(g, g)))
    W, H = fh.iteration(A, w[:, None].copy(), H0.astype(np.float64), EPS)
    assert np.allclose(H[0], h1, rtol=1e-12, atol=0)
    assert np.allclose(W[:, 0], w1, rtol=1e-12, atol=0)


def test_k1_limit_is_perron_vector():
    """The K = 1 iteration is a power iteration on A A^T: w -> u1, h -> s1 v1,
    objective -> ||A||^2 - s1^2 (LAPACK SVD)."""
    A = _dense(40, 30, 3, 2)
    W0, H0 = synth.init_factors(3, 40, 30, 1)
    W, H, _ = fh.run(A, W0, H0, 200)
    U, s, Vt = np.linalg.svd(A)
    u1 = np.abs(U[:, 0])
    assert np.max(np.abs(W[:, 0] - u1)) < 1e-10
    assert np.max(np.abs(H[0] - s[0] * np.abs(Vt[0]))) < 1e-10 * s[0]
    f_expected = float(np.sum(A * A)) - s[0] ** 2
    assert abs(ob.frob2_direct(A, W, H) - f_expected) <= 1e-10 * float(np.sum(A * A))


# --- planted exact recovery ----------------------------------------------------

def test_planted_separable_recovery():
    rng = np.random.default_rng(0)
    V, D, K = 12, 10, 3
    W0 = np.zeros((V, K))
    for v in range(V):
        W0[v, v % K] = 0.5 + rng.random()
    # H0 holds an identity block and zeros, so the exact NMF is unique up to
    # permutation and scaling of the columns of W
    H0 = (0.5 + rng.random((K, D))) * (rng.random((K, D)) < 0.5)
    H0[:, :K] = np.eye(K)
    A = W0 @ H0
    Wi, Hi = synth.init_factors(11, V, D, K)
    W, H, _ = fh.run(A, Wi, Hi, 600)
    assert ob.relative_error(A, W, H, direct=True) < 1e-8
    # factors match up to permutation and scale: each recovered column is
    # proportional to one planted column
    Wn = W0 / np.linalg.norm(W0, axis=0)
    C = np.abs(W.T @ Wn)
    assert np.allclose(np.sort(C.max(axis=1)), 1.0, atol=1e-8)
    assert sorted(C.argmax(axis=1).tolist()) == [0, 1, 2]


# --- KKT -----------------------------------------------------------------------

def test_kkt_residual_decays():
    A = _dense(64, 48, 4, 13)
    W0, H0 = synth.init_factors(14, 64, 48, 4)
    W, H = fh.normalize_init(W0), H0.astype(np.float64)

    def kkt(W, H):
        gW = W @ (H @ H.T) - A @ H.T
        gH = (W.T @ W) @ H - W.T @ A
        return math.hypot(np.linalg.norm(np.minimum(W - EPS, gW)),
                          np.linalg.norm(np.minimum(H - EPS, gH)))

    W, H = fh.iteration(A, W, H, EPS)
    k0 = kkt(W, H)
    for _ in range(1500):
        W, H = fh.iteration(A, W, H, EPS)
    assert kkt(W, H) < 1e-4 * k0


# --- Eq. 2 directly vs the trace identity -------------------------------------

def test_trace_identity_dense_and_sparse():
    A = _dense(50, 40, 5, 17)
    W0, H0 = synth.init_factors(18, 50, 40, 6)
    W, H, _ = fh.run(A, W0, H0, 3)
    a, b = ob.frob2_direct(A, W, H), ob.frob2_trace(A, W, H)
    assert abs(a - b) <= 1e-10 * a
    sp = synth.sparse_termdoc(500, 200, 19, mean_terms=25)
    W0, H0 = synth.init_factors(20, 500, 200, 8)
    W, H, _ = fh.run(sp.A, W0, H0, 3)
    a, b = ob.frob2_direct(sp.A, W, H), ob.frob2_trace(sp.A, W, H)
    assert abs(a - b) <= 1e-10 * a
    # ||A||_F^2 = D for column-normalised tf-idf
    assert abs(ob.norm2_A(sp.A) - 200) < 1e-4


# --- fixed-W H subproblem ------------------------------------------------------

def test_fixed_w_sweeps_reach_nnls_optimum():
    rng = np.random.default_rng(5)
    V, K = 30, 6
    W = np.abs(rng.normal(size=(V, K)))
    W /= np.linalg.norm(W, axis=0)
    docs = np.abs(rng.normal(size=(V, 5))) * (rng.random((V, 5)) < 0.5)
    Rt = docs.T @ W
    S = W.T @ W
    H, sweeps = nnls.hals_sweeps(Rt, S, np.full((K, 5), 0.5), EPS, tol=1e-14)
    for j in range(5):
        x_lh = nnls.nnls_lawson_hanson(W, docs[:, j])
        x_bf = nnls.nnls_bruteforce(W, docs[:, j])
        assert np.allclose(x_lh, x_bf, atol=1e-10)
        assert np.allclose(H[:, j], x_bf, atol=1e-9)


# --- warm-start network: analytic gradients vs central differences ------------

def test_mlp_gradients_finite_difference():
    rng = np.random.default_rng(1)
    sizes = [(7, 9), (9, 9), (9, 5)]
    params = []
    for (i, o) in sizes:
        params += [rng.normal(scale=0.5, size=(i, o)), rng.normal(scale=0.1, size=o)]
    x = rng.normal(size=(4, 7))
    t = np.abs(rng.normal(size=(4, 5)))
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        for j in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[j]
            flat[j] = old + h
            lp = mlp.loss(params, x, t)
            flat[j] = old - h
            lm = mlp.loss(params, x, t)
            flat[j] = old
            num = (lp - lm) / (2 * h)
            ana = grads[pi].reshape(-1)[j]
            assert abs(num - ana) <= 1e-7 * max(1.0, abs(ana)) + 1e-9


def test_mlp_operand_rounding_is_exact_on_representable_operands():
    """The reduced-precision-product form rounds only product operands: a
    network whose input, weights and hidden activations are all exactly
    representable in BF16 gives the same output with and without rounding
    (x and weights are small dyadic numbers; zero first-layer weights make
    a1 = GELU(b1) with b1 = 0 -> a1 = 0, and W2 = 0 makes a2 = GELU(0) = 0),
    while generic operands move the output by about the BF16 unit roundoff
    (2^-8 relative per operand; bounded over three layers)."""
    from oracle.bf16 import round_bf16
    rng = np.random.default_rng(3)
    x = rng.integers(-4, 5, size=(6, 5)) / 4.0
    params = [np.zeros((5, 8)), np.zeros(8), np.zeros((8, 8)), np.zeros(8),
              rng.integers(-3, 4, size=(8, 5)) / 8.0, rng.integers(-3, 4, size=5) / 8.0]
    y0, _ = mlp.forward(params, x)
    y1, _ = mlp.forward(params, x, operand_round=round_bf16)
    assert np.array_equal(y0, y1)
    # generic operands: a change that is present but BF16-sized
    params = []
    for (i, o) in [(5, 8), (8, 8), (8, 5)]:
        params += [rng.normal(scale=0.5, size=(i, o)), rng.normal(scale=0.1, size=o)]
    x = rng.normal(size=(6, 5))
    t = np.abs(rng.normal(size=(6, 5)))
    y0, c0 = mlp.forward(params, x)
    y1, c1 = mlp.forward(params, x, operand_round=round_bf16)
    d = np.linalg.norm(y1 - y0) / np.linalg.norm(y0)
    assert 1e-5 < d < 6 * 2.0 ** -8
    g0 = mlp.backward(params, c0, y0, t)
    g1 = mlp.backward(params, c1, y1, t, operand_round=round_bf16)
    for a, b in zip(g0, g1):
        assert np.linalg.norm(a - b) <= 12 * 2.0 ** -8 * np.linalg.norm(a)


def test_mlp_activation_closed_forms():
    # GELU(0) = 0, GELU(x) -> x for large x, softplus(0) = ln 2, threshold branch.
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(10.0)) - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15   # Phi(1) = 0.84134...
    assert abs(mlp.softplus(np.array(0.0)) - math.log(2.0)) < 1e-15
    assert mlp.softplus(np.array(25.0)) == 25.0


def test_adam_first_step_is_sign_times_lr():
    # With bias correction the first Adam step is lr * g / (|g| + eps').
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    out, m, v = mlp.adam_step(p, g, [np.zeros(3)], [np.zeros(3)], 1, lr=0.1)
    assert np.allclose(out[0], p[0] - 0.1 * g[0] / (np.abs(g[0]) + 1e-8), atol=1e-15)


# --- the paper's printed model numbers (Sec. 5) --------------------------------

def test_paper_worked_numbers():
    g = _golden("paper_worked_numbers.txt")
    C = tm.CACHE_35MB_WORDS
    assert tm.fast_hals_w_loop(11314, 160) == g["w_loop_words_V11314_K160"]
    assert math.floor(tm.vol(11314, 160, 15, C)) == g["plnmf_vol_V11314_K160_T15"]
    for K, key in ((80, "tile_K80"), (160, "tile_K160"), (240, "tile_K240")):
        # the paper prints the values truncated to two decimals
        assert math.floor(tm.tile_size_printed(K, C) * 100) / 100 == pytest.approx(g[key], abs=1e-9)
        # the exact stationary point of Eq. 9 rounds to the same tile sizes
        assert abs(tm.tile_size_stationary(K, C) - g[key]) < 0.02
    ratio = tm.fast_hals_w_loop(11314, 160) / tm.vol(11314, 160, 15, C)
    assert round(ratio, 1) == g["reduction_factor"]


# --- planted mistakes: each pin above catches a plausible oracle bug ----------

def test_pins_catch_planted_mistakes(monkeypatch):
    A = _dense(40, 30, 3, 2)
    W0, H0 = synth.init_factors(3, 40, 30, 5)

    # (1) Jacobi instead of Gauss-Seidel in the H loop -> reorder pin fails.
    def jacobi_h(R, S, H, eps=EPS):
        H = np.array(H, dtype=np.float64)
        return np.maximum(eps, H + R.T - S.T @ H)
    W = fh.normalize_init(W0)
    tr = {}
    monkeypatch.setattr(fh, "update_h", jacobi_h)
    W1, H1 = fh.iteration(A, W, H0, EPS, trace=tr)
    monkeypatch.undo()
    Hp = pl_nmf.update_h(tr["R"], tr["S"], H0, 2, EPS)
    assert np.max(np.abs(Hp - H1)) > 1e-6

    # (2) sign error on P in the W loop -> monotone pin fails.
    def bad_w(P, Q, W, eps=EPS):
        W = np.array(W, dtype=np.float64)
        for k in range(W.shape[1]):
            W[:, k] = np.maximum(eps, W[:, k] * Q[k, k] - P[:, k] - W @ Q[:, k])
            W[:, k] /= np.linalg.norm(W[:, k])
        return W
    monkeypatch.setattr(fh, "update_w", bad_w)
    W, H = fh.normalize_init(W0), H0.astype(np.float64)
    fs = []
    for _ in range(6):
        W, H = fh.iteration(A, W, H, EPS)
        fs.append(ob.frob2_direct(A, W, H))
    monkeypatch.undo()
    assert any(b > a * (1 + 1e-12) for a, b in zip(fs, fs[1:])) or fs[-1] > fs[0] * 0.9

    # (3) dropped normalisation -> K = 1 closed form fails.
    def unnormalised_w(P, Q, W, eps=EPS):
        W = np.array(W, dtype=np.float64)
        for k in range(W.shape[1]):
            W[:, k] = np.maximum(eps, W[:, k] * Q[k, k] + P[:, k] - W @ Q[:, k])
        return W
    monkeypatch.setattr(fh, "update_w", unnormalised_w)
    w = fh.normalize_init(W0[:, :1])
    Wb, _ = fh.iteration(A, w, H0[:1].astype(np.float64), EPS)
    monkeypatch.undo()
    assert abs(np.linalg.norm(Wb[:, 0]) - 1.0) > 1e-3


# --- BF16 rounding (operands of the BF16 form) ---------------------------------

def test_round_bf16_definition_and_library_agree():
    import torch
    from oracle.bf16 import round_bf16
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-6, 6, size=20000),
                        np.array([0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, 65504.0])])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(round_bf16(x), ref)
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1
    assert round_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert round_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6


def test_round_bf16_split_bound_exactness_and_library():
    """The BF16 pair (hi, lo) of the split form: exact for values whose binary32
    significand fits in the two BF16 significands, within 2^-16 |x| always,
    and hi, lo are the library's BF16 roundings of x and of x - hi."""
    import torch
    from oracle.bf16 import round_bf16, round_bf16_split
    rng = np.random.default_rng(11)
    # exactly representable pairs: an 8-bit significand plus one 8 binades lower
    hi = round_bf16(rng.random(4000) + 0.5)
    # |lo| in [2^-11, 2^-10): below half a BF16 ulp of hi, and hi + lo spans
    # at most 19 significant bits
    lo = round_bf16(np.where(rng.random(4000) < 0.5, -1.0, 1.0) * (1.0 + rng.random(4000)) * 2.0 ** -11)
    x = (hi + lo).astype(np.float32).astype(np.float64)
    assert np.array_equal(x, hi + lo)                    # the pair is a binary32 value
    assert np.array_equal(round_bf16_split(x), x)
    # bound on arbitrary binary32 values over many binades
    y = (rng.random(200000) * 10.0 ** rng.integers(-8, 8, size=200000)).astype(np.float32).astype(np.float64)
    err = np.abs(round_bf16_split(y) - y)
    assert np.all(err <= 2.0 ** -16 * np.abs(y))
    assert np.max(err / y) > 2.0 ** -20                  # not exact in general: the bound is not vacuous
    # the two parts against the library's conversion
    t = torch.from_numpy(y.astype(np.float32))
    th = t.to(torch.bfloat16).to(torch.float32)
    tl = (t - th).to(torch.bfloat16).to(torch.float64)
    assert np.array_equal(round_bf16_split(y), th.double().numpy() + tl.numpy())
    # planted mistake: lo rounded from x instead of from x - hi breaks the bound
    bad = round_bf16(y) + round_bf16(y)
    assert np.max(np.abs(bad - y) / y) > 0.5


def test_adam_later_steps_match_expanded_moments():
    """Adam over four steps with varying gradients against the moments
    written out as weighted sums, m_t = (1 - b1) sum_s b1^(t-s) g_s and
    v_t = (1 - b2) sum_s b2^(t-s) g_s^2, each step p -= lr mhat / (sqrt(vhat) + eps).
    An oracle that failed to carry m or v between steps passes the first
    step (where the step is lr g / (|g| + eps) whatever they hold) but not this."""
    b1, b2, lr, eps = 0.9, 0.999, 0.05, 1e-8
    gs = [np.array([0.5, -4.0, 1e-3]), np.array([-1.0, 2.0, 3.0]), np.array([0.25, 0.0, -2.0]),
          np.array([2.0, -1.0, 0.5])]
    p = [np.array([1.0, -2.0, 3.0])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    expect = np.array([1.0, -2.0, 3.0])
    for t in range(1, len(gs) + 1):
        p, m, v = mlp.adam_step(p, [gs[t - 1]], m, v, t, lr=lr, b1=b1, b2=b2, eps=eps)
        mt = (1 - b1) * sum(b1 ** (t - s) * gs[s - 1] for s in range(1, t + 1))
        vt = (1 - b2) * sum(b2 ** (t - s) * gs[s - 1] ** 2 for s in range(1, t + 1))
        expect = expect - lr * (mt / (1 - b1 ** t)) / (np.sqrt(vt / (1 - b2 ** t)) + eps)
        assert np.allclose(m[0], mt, rtol=1e-14, atol=1e-16)
        assert np.allclose(v[0], vt, rtol=1e-14, atol=1e-16)
        assert np.allclose(p[0], expect, rtol=1e-13, atol=1e-15)
    # planted mistake: moments restarted every step -> the fourth parameter set differs
    q = [np.array([1.0, -2.0, 3.0])]
    for t in range(1, len(gs) + 1):
        q, _, _ = mlp.adam_step(q, [gs[t - 1]], [np.zeros(3)], [np.zeros(3)], t, lr=lr, b1=b1, b2=b2, eps=eps)
    assert np.max(np.abs(q[0] - expect)) > 1e-3


def test_operand_rounding_hook_is_identity_when_unset():
    A = _dense(30, 20, 3, 4)
    W0, H0 = synth.init_factors(5, 30, 20, 4)
    W, H = fh.normalize_init(W0), H0.astype(np.float64)
    a = fh.iteration(A, W, H, EPS)
    b = fh.iteration(A, W, H, EPS, operand_round=lambda x: x)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# --- multiplicative updates (MU comparator) ---------------------------------

def test_mu_k1_h_step_is_least_squares():
    """K = 1: one MU H step gives h_j = w^T a_j / w^T w for every positive
    h_j, the unconstrained least-squares minimiser (non-negative for A >= 0)."""
    from oracle import mu
    rng = np.random.default_rng(3)
    A = rng.random((40, 30))
    w = rng.random((40, 1))
    h0 = rng.random((1, 30)) + 0.1
    h1 = mu.update_h(A, w, h0, delta=0.0)
    np.testing.assert_allclose(h1[0], (w[:, 0] @ A) / (w[:, 0] @ w[:, 0]), rtol=1e-13)


def test_mu_exact_factorisation_is_fixed_point():
    from oracle import mu
    rng = np.random.default_rng(4)
    W = rng.random((50, 6)) + 0.05
    H = rng.random((6, 35)) + 0.05
    A = W @ H
    W1, H1 = mu.iteration(A, W, H, delta=0.0)
    np.testing.assert_allclose(H1, H, rtol=1e-12)
    np.testing.assert_allclose(W1, W, rtol=1e-12)


def test_mu_objective_non_increasing_and_order():
    """Lee & Seung's monotonicity, on dense and sparse inputs; and the order
    of the two updates (H first, with the current W) matters."""
    from oracle import mu
    for A in (synth.planted_dense(60, 45, 5, 9).A.astype(np.float64),
              synth.sparse_termdoc(300, 120, 5, mean_terms=12).A):
        V, D = (A.n_rows, A.n_cols) if hasattr(A, "n_rows") else A.shape
        W0, H0 = synth.init_factors(11, V, D, 4)
        W, H = mu.normalize_init(W0), H0.astype(np.float64)
        f_prev = np.inf
        for _ in range(30):
            W, H = mu.iteration(A, W, H)
            f = ob.frob2_direct(A, W, H)
            assert f <= f_prev * (1 + 1e-12)
            f_prev = f
    A = synth.planted_dense(60, 45, 5, 9).A.astype(np.float64)
    W0, H0 = synth.init_factors(12, 60, 45, 4)
    W, H = mu.normalize_init(W0), H0.astype(np.float64)
    Wa, Ha = mu.iteration(A, W, H)
    Wb = mu.update_w(A, W, H)                          # W first: a different iterate
    assert not np.allclose(Wa, Wb)
