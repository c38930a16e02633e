"""BF16 precision form (dense A): tensor-core products and Grams with BF16
operands, FP32 updates, objective against the FP32 A.

Oracle: Alg. 1 with the operands of its four products rounded to BF16 and
everything else FP64 (oracle.fast_hals.iteration(operand_round=round_bf16)).
On the planted test matrices (rank = K) the first W update is nearly
singular: the FP64 oracle itself moves W by ~0.3 when only its product
operands are rounded to BF16, so W is compared with the BF16-operand oracle
and H (well conditioned) also with the plain FP64 oracle.  Tolerances: one
iteration 2e-2 (max-norm relative); objective after 100 iterations on
planted inputs: see test_objective_after_100_iterations_against_oracle."""

import math

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle import objective as ob
from oracle.bf16 import round_bf16
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
    ctx = _ctx(nmf, prob.A, 48, W0, H0)
    ctx.iterate(1)
    Wg, Hg = ctx.get_factors()
    start = (fh.normalize_init(W0), H0.astype(np.float64))
    Wb, Hb = fh.iteration(prob.A, *start, EPS, operand_round=round_bf16)
    Wr, Hr = fh.iteration(prob.A, *start, EPS)
    assert rel_h(Hg, Hb) < 2e-2 and rel_w(Wg, Wb) < 2e-2
    assert rel_h(Hg, Hr) < 2e-2


@pytest.mark.parametrize("shape", [(1024, 768, 8), (512, 384, 16)])
def test_objective_after_100_iterations_against_oracle(nmf, shape):
    """Relative objective after 100 iterations on planted rank-r inputs
    (rank r = K).  FP32 form: within 1e-4 of the FP64 oracle.  BF16 form:
    within 3e-3 of the BF16-operand oracle (its definition, Alg. 1 with the
    product operands rounded to BF16): separate orderings of the same BF16
    arithmetic scatter by about 1e-3 over 100 unconverged iterations
    (measured: -1.1e-3 .. +1.0e-3 over three inputs, while the FP64 and
    BF16-operand oracles themselves differ by 1e-3 .. 4e-3 there).  nmf_error
    measures the fit to the FP32 A, not to its BF16 copy."""
    import torch
    V, D, r = shape
    prob = synth.planted_dense(V, D, r, 0xC3 + 7)
    A = prob.A
    W0, H0 = synth.init_factors(9, V, D, r)
    Wr, Hr, _ = fh.run(A, W0, H0, 100)
    f64 = ob.frob2_direct(A, Wr, Hr)
    Wb, Hb, _ = fh.run(A, W0, H0, 100, operand_round=round_bf16)
    fb = ob.frob2_direct(A, Wb, Hb)
    for prec, ref, tol in ((nmf.PREC_FP32, f64, 1e-4), (nmf.PREC_BF16, fb, 3e-3)):
        ctx = nmf.from_dense(A, r, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(), prec=prec)
        ctx.iterate(100)
        f_gpu, rel = ctx.error()
        Wg, Hg = ctx.get_factors()
        f_direct = ob.frob2_direct(A, Wg, Hg)
        assert abs(f_gpu - f_direct) <= 1e-5 * f_direct
        assert abs(rel - math.sqrt(f_direct / ob.norm2_A(A))) <= 1e-5
        assert abs(f_direct - ref) <= tol * ref, (prec, f_direct, ref)


def test_bf16_rejected_for_sparse(nmf):
    sp = synth.sparse_termdoc(300, 200, 5, mean_terms=10)
    with pytest.raises(nmf.NmfError) as e:
        nmf.from_sparse(sp, 8, prec=nmf.PREC_BF16)
    assert e.value.status == nmf.NMF_EUNSUPPORTED


# --- the TMA-fed BF16 product (Alg. 1 lines 4 and 10 of the BF16 form) -----

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
    """The two tensor-core paths of the BF16 form compute the same products
    (BF16 operands, FP32 accumulation) in different summation orders."""
    import torch
    prob = synth.planted_dense(700, 530, 40, 0xC3 + 2)
    W0, H0 = synth.init_factors(11, 700, 530, 40)
    out = []
    for flags in (0, nmf.FLAG_NO_TMA):
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
