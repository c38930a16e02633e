"""Tensor-core GEMM (tcgen05, 3xTF32 and BF16) against an FP64 product, via
the C-ABI utility nmf_gemm, on ragged shapes that span several tiles."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf
    return torch, nmf


SHAPES = [(128, 32, 32, False), (300, 37, 77, False), (160, 160, 700, True), (257, 130, 96, True),
          (64, 256, 512, False), (1000, 160, 33, False)]


@pytest.mark.parametrize("M,N,K,transA", SHAPES)
def test_tf32x3_matches_fp64(env, M, N, K, transA):
    torch, nmf = env
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.random((K, M) if transA else (M, K), dtype=np.float64).astype(np.float32)
    B = rng.random((K, N), dtype=np.float64).astype(np.float32)
    C = torch.full((M, N), float("nan"), device="cuda")
    nmf.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, transA=transA, prec=nmf.PREC_FP32)
    torch.cuda.synchronize()
    ref = (A.astype(np.float64).T if transA else A.astype(np.float64)) @ B.astype(np.float64)
    got = C.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    # 3xTF32 split error (~2^-21 per product) plus the tensor core's FP32
    # accumulation, which truncates: up to ~2^-24 per added term.
    assert err < K * 2.0 ** -24 + 2.0 ** -21, err


@pytest.mark.parametrize("M,N,K,transA", SHAPES[:4])
def test_bf16_products(env, M, N, K, transA):
    torch, nmf = env
    rng = np.random.default_rng(11 + M + N + K)
    A = rng.random((K, M) if transA else (M, K), dtype=np.float64).astype(np.float32)
    B = rng.random((K, N), dtype=np.float64).astype(np.float32)
    C = torch.zeros((M, N), device="cuda")
    nmf.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, transA=transA, prec=nmf.PREC_BF16)
    torch.cuda.synchronize()
    # reference with the operands rounded to BF16 exactly as the kernel does
    bf = lambda x: torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    Ab = bf(A)
    ref = (Ab.T if transA else Ab) @ bf(B)
    got = C.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-5


def test_tc_grams_option_close_to_simt(env):
    """The opt-in tensor-core Grams agree with the SIMT FP32 Grams within the
    truncated-accumulation bound."""
    torch, nmf = env
    from paper_1904_07935_b300 import synth
    sp = synth.sparse_termdoc(3000, 1400, 5, mean_terms=40)
    W0, H0 = synth.init_factors(6, 3000, 1400, 48)
    a = nmf.from_sparse(sp, 48, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda())
    b = nmf.from_sparse(sp, 48, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(),
                        flags=nmf.FLAG_TC_GRAMS)
    for c in (a, b):
        c.run_step(nmf.STEP_S)
        c.run_step(nmf.STEP_Q)
    for which, n in ((nmf.BUF_S, 3000), (nmf.BUF_Q, 1400)):
        sa, sb = a.get_buffer(which), b.get_buffer(which)
        assert np.max(np.abs(sa - sb)) / np.max(np.abs(sa)) < 352 * 2.0 ** -24 + 2.0 ** -20
