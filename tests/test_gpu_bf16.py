"""BF16 precision form (dense A): tensor-core products and Grams with BF16
operands, FP32 updates, objective against the FP32 A.

Every tensor-core operand is carried as a BF16 pair x = x_hi + x_lo (x_hi =
bf16(x), x_lo = bf16(x - x_hi), about 16 significant bits) and each product
is the sum of three BF16 MMAs with FP32 accumulation.  Oracle: Alg. 1 with the
operands of its four products carried as such pairs and everything else FP64
(oracle.fast_hals.iteration(operand_round=round_bf16_split)); the forms that
round the factors (NMF_FLAG_BF16_SINGLE_FACTORS) or A as well
(NMF_FLAG_BF16_SINGLE_A) to BF16 once are checked against their own
definitions.  Tolerances (the benchmark spec): one iteration 2e-2 max-norm relative;
relative objective after 100 iterations 1e-3 against the FP64 oracle.

From a random start the planted rank-K inputs are chaotic over 100 iterations:
the FP64 oracle itself, started from W0 perturbed by one FP32 unit in the
last place, ends 2.4% away in objective at 2048 x 2048, K = 256 (measured), so
no reduced-precision arithmetic can be held to 1e-3 there; that size is
checked from the oracle's iterate 100, where the oracle is stable.  The first
W update from a random start is ill-conditioned on the same inputs (r18 of
the design notes), so one-iteration W parity is taken from iterate 10.
"""

import math

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle import objective as ob
from oracle.bf16 import round_bf16, round_bf16_split
from paper_1904_07935_b300 import synth

from ._parity import rel_h, rel_w

pytestmark = pytest.mark.gpu

EPS = 1e-16


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


def _ctx(nmf, A, K, W0, H0):
    import torch
    return nmf.from_dense(A, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(),
                          prec=nmf.PREC_BF16)


def test_bf16_one_iteration(nmf):
    prob = synth.planted_dense(1000, 780, 48, 0xC3)      # ragged against 128-row tiles
    W0, H0 = synth.init_factors(7, 1000, 780, 48)
    # random start: H (well conditioned) against both oracles
    ctx = _ctx(nmf, prob.A, 48, W0, H0)
    ctx.iterate(1)
    _, Hg = ctx.get_factors()
    start = (fh.normalize_init(W0), H0.astype(np.float64))
    _, Hx = fh.iteration(prob.A, *start, EPS, operand_round=round_bf16_split)
    _, Hr = fh.iteration(prob.A, *start, EPS)
    assert rel_h(Hg, Hx) < 2e-2 and rel_h(Hg, Hr) < 2e-2
    # from the oracle's iterate 10: W and H (measured 4.8e-3 / 2.6e-6)
    W10, H10, _ = fh.run(prob.A, W0, H0, 10)
    W10, H10 = W10.astype(np.float32), H10.astype(np.float32)
    ctx = _ctx(nmf, prob.A, 48, W10, H10)
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    start = (fh.normalize_init(W10), H10.astype(np.float64))
    Wx, Hx = fh.iteration(prob.A, *start, EPS, operand_round=round_bf16_split)
    Wr, Hr = fh.iteration(prob.A, *start, EPS)
    for W, H in ((Wx, Hx), (Wr, Hr)):
        assert rel_w(Wg, W) < 2e-2 and rel_h(Hg, H) < 2e-2


@pytest.mark.parametrize("shape", [(1024, 768, 8), (512, 384, 16)])
def test_objective_after_100_iterations_against_oracle(nmf, shape):
    """Relative objective after 100 iterations on planted rank-r inputs
    (rank r = K), random start.  FP32 form within 1e-4 and BF16 form within
    1e-3 of the FP64 oracle (measured: 2e-6 / 9e-6 and 8e-5 / 1.3e-5).  The
    form with A and the factors rounded to BF16 once is held to its own
    definition (the BF16-operand oracle) at 3e-3: separate orderings of that
    arithmetic scatter by about 1e-3 over 100 unconverged iterations.
    nmf_error measures the fit to the FP32 A, not to its BF16 copy."""
    import torch
    V, D, r = shape
    prob = synth.planted_dense(V, D, r, 0xC3 + 7)
    A = prob.A
    W0, H0 = synth.init_factors(9, V, D, r)
    Wr, Hr, _ = fh.run(A, W0, H0, 100)
    f64 = ob.frob2_direct(A, Wr, Hr)
    Wb, Hb, _ = fh.run(A, W0, H0, 100, operand_round=round_bf16)
    fb = ob.frob2_direct(A, Wb, Hb)
    for prec, flags, ref, tol in ((nmf.PREC_FP32, 0, f64, 1e-4), (nmf.PREC_BF16, 0, f64, 1e-3),
                                  (nmf.PREC_BF16, nmf.FLAG_BF16_SINGLE_A, fb, 3e-3)):
        ctx = nmf.from_dense(A, r, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(), prec=prec,
                             flags=flags)
        ctx.iterate(100)
        f_gpu, rel = ctx.error()
        Wg, Hg = ctx.get_factors()
        f_direct = ob.frob2_direct(A, Wg, Hg)
        assert abs(f_gpu - f_direct) <= 1e-5 * f_direct
        assert abs(rel - math.sqrt(f_direct / ob.norm2_A(A))) <= 1e-5
        assert abs(f_direct - ref) <= tol * ref, (prec, flags, f_direct, ref)


def test_objective_2048_k256_against_fp64_oracle(nmf):
    """Planted rank-256 2048 x 2048 input, K = 256: 100 iterations from the
    FP64 oracle's iterate 100 (where the oracle is stable: one FP32 ulp on the
    start moves its objective by 4e-9).  FP32 form within 1e-4 and BF16 form
    within 1e-3 of the FP64 oracle (measured 8e-7 and 5.5e-4)."""
    import torch
    prob = synth.planted_dense(2048, 2048, 256, 0xC3 + 9)
    A = prob.A
    W0, H0 = synth.init_factors(9, 2048, 2048, 256)
    Ws, Hs, _ = fh.run(A, W0, H0, 100)
    Ws, Hs = Ws.astype(np.float32), Hs.astype(np.float32)
    Wr, Hr, _ = fh.run(A, Ws, Hs, 100)
    f64 = ob.frob2_direct(A, Wr, Hr)
    for prec, tol in ((nmf.PREC_FP32, 1e-4), (nmf.PREC_BF16, 1e-3)):
        ctx = nmf.from_dense(A, 256, W0=torch.from_numpy(Ws).cuda(), H0=torch.from_numpy(Hs).cuda(), prec=prec)
        ctx.iterate(100)
        Wg, Hg = ctx.get_factors()
        f_direct = ob.frob2_direct(A, Wg, Hg)
        assert abs(f_direct - f64) <= tol * f64, (prec, f_direct, f64)


def test_bf16_rejected_for_sparse(nmf):
    sp = synth.sparse_termdoc(300, 200, 5, mean_terms=10)
    with pytest.raises(nmf.NmfError) as e:
        nmf.from_sparse(sp, 8, prec=nmf.PREC_BF16)
    assert e.value.status == nmf.NMF_EUNSUPPORTED


# --- the TMA-fed BF16 product (R = A^T W and P = A H^T of Alg. 1, BF16 form)

def _bf16_bound(a64, b64):
    """|C - A B^T| bound: BF16 x BF16 products are exact in FP32, so only the
    FP32 accumulation rounds (<= K * 2^-23 relative to sum |a||b| for any
    order or truncating adds), plus an absolute floor."""
    K = a64.shape[1]
    return (K * 2.0 ** -23) * (np.abs(a64) @ np.abs(b64).T) + 2.0 ** -40


@pytest.mark.parametrize("M,N,K,pad", [(128, 128, 64, 0), (300, 200, 1000, 0), (129, 256, 4104, 8),
                                       (1000, 160, 777 + 7, 16), (8, 8, 8, 0)])
def test_gemm_bf16_tma_against_fp64(nmf, M, N, K, pad):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    lda = (K + 7) // 8 * 8 + pad
    Ab = torch.zeros(M, lda, dtype=torch.bfloat16)
    Bb = torch.zeros(N, lda, dtype=torch.bfloat16)
    Ab[:, :K] = torch.rand(M, K, generator=g).to(torch.bfloat16)
    Bb[:, :K] = (torch.randn(N, K, generator=g)).to(torch.bfloat16)
    # garbage beyond K in the padded stride must not enter the product
    if lda > K:
        Ab[:, K:] = 1e30
        Bb[:, K:] = -1e30
    C = torch.full((M, N + 3), float("nan"), device="cuda")[:, :N]
    nmf.gemm_bf16(Ab.cuda()[:, :K], Bb.cuda()[:, :K], C)     # row stride lda, K columns
    torch.cuda.synchronize()
    a64 = Ab[:, :K].double().numpy()
    b64 = Bb[:, :K].double().numpy()
    ref = a64 @ b64.T
    err = np.abs(C.cpu().double().numpy() - ref)
    assert np.all(err <= _bf16_bound(a64, b64))


def test_gemm_bf16_tma_rejects_bad_strides(nmf):
    import torch
    A = torch.zeros(64, 20, dtype=torch.bfloat16, device="cuda")     # lda = 20, not a multiple of 8
    B = torch.zeros(64, 24, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(64, 64, device="cuda")
    with pytest.raises(nmf.NmfError) as e:
        nmf.gemm_bf16(A, B[:, :20], C)
    assert e.value.status == nmf.NMF_EINVAL


def test_bf16_form_tma_matches_staged_kernel(nmf):
    """With A rounded to BF16 once, the two tensor-core paths of the BF16 form
    compute the same products (BF16 operands, FP32 accumulation) in different
    summation orders."""
    import torch
    prob = synth.planted_dense(700, 530, 40, 0xC3 + 2)
    W0, H0 = synth.init_factors(11, 700, 530, 40)
    out = []
    for flags in (nmf.FLAG_BF16_SINGLE_A, nmf.FLAG_NO_TMA):
        ctx = nmf.from_dense(prob.A, 40, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(),
                             prec=nmf.PREC_BF16, flags=flags)
        ctx.run_step(nmf.STEP_R)
        R = ctx.get_buffer(nmf.BUF_R)
        ctx.run_step(nmf.STEP_P)
        P = ctx.get_buffer(nmf.BUF_P)
        out.append((R, P))
    for x, y in zip(out[0], out[1]):
        # nonnegative operands: sum |a||b| = the product; FP32 accumulation of
        # <= 700 terms in either order moves it by at most 700 * 2^-23 relative
        assert np.max(np.abs(x - y)) <= 700 * 2.0 ** -23 * np.max(np.abs(y))


def _split_ctx(nmf, prob, K, W0, H0, flags):
    import torch
    return nmf.from_dense(prob.A, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(),
                          prec=nmf.PREC_BF16, flags=flags)


def test_bf16_split_products_against_fp64(nmf):
    """R = A^T W and P = A H^T of the BF16 form against FP64 products.  Every
    operand a BF16 pair (default): against the exact A and factor the error is
    the pairs' representation error (<= 2^-16 per operand, plus the omitted
    lo x lo term, <= 2^-18) plus FP32 accumulation (<= L 2^-23), relative to
    sum |a||f|.  Factors rounded once: against A times the rounded factor,
    2^-16 + L 2^-23.  A rounded once as well misses that reference by far
    more (its 2^-9 error)."""
    V, D, K = 777, 650, 40
    prob = synth.planted_dense(V, D, 24, 0xC3 + 3)
    W0, H0 = synth.init_factors(13, V, D, K)
    A = prob.A.astype(np.float64)
    outs = {}
    for flags in (0, nmf.FLAG_BF16_SINGLE_FACTORS, nmf.FLAG_BF16_SINGLE_A):
        ctx = _split_ctx(nmf, prob, K, W0, H0, flags)
        W = ctx.get_buffer(nmf.BUF_W).astype(np.float64)
        Ht = ctx.get_buffer(nmf.BUF_HT).astype(np.float64)
        ctx.run_step(nmf.STEP_R)
        R = ctx.get_buffer(nmf.BUF_R)
        ctx.run_step(nmf.STEP_P)
        outs[flags] = (R, ctx.get_buffer(nmf.BUF_P), W, Ht)
    R, P, W, Ht = outs[0]
    for got, Aop, F, L in ((R, A.T, W, V), (P, A, Ht, D)):
        bound = (2 * 2.0 ** -16 + 2.0 ** -18 + L * 2.0 ** -23) * (np.abs(Aop) @ np.abs(F)) + 2.0 ** -40
        assert np.all(np.abs(got - Aop @ F) <= bound)
    R, P, W, Ht = outs[nmf.FLAG_BF16_SINGLE_FACTORS]
    for got, Aop, F, L in ((R, A.T, round_bf16(W), V), (P, A, round_bf16(Ht), D)):
        bound = (2.0 ** -16 + L * 2.0 ** -23) * (np.abs(Aop) @ np.abs(F)) + 2.0 ** -40
        assert np.all(np.abs(got - Aop @ F) <= bound)
    Ps = outs[nmf.FLAG_BF16_SINGLE_A][1]
    ref = A @ round_bf16(Ht)
    assert np.max(np.abs(Ps - ref)) > 20 * np.max(np.abs(P - ref))
