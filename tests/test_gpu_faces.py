"""Dense face-image-shaped workloads (the shapes of the paper's AT&T and PIE
datasets, Table 4; synthetic contents from `synth.faces_like`): one
iteration on the GPU against the FP64 oracle at full size.

The first W updates of these near-square factorisations (AT&T: 400 images)
cancel heavily, so each case starts from an early oracle iterate where the
FP32 storage floor d32 (`fp32_storage_sensitivity`) is below 3e-6, checked
in the test, and holds the strict 1e-5.  The BF16 form is compared with its
definition, Alg. 1 with the operands of its products carried as BF16 pairs
(hi = bf16(x), lo = bf16(x - hi)), within 2e-2."""

import numpy as np
import pytest

from oracle import fast_hals as fh
from oracle.bf16 import round_bf16_split
from paper_1904_07935_b300 import synth

from ._parity import f32, fp32_storage_sensitivity, rel_h, rel_w

pytestmark = pytest.mark.gpu

EPS = 1e-16
TOL_ITER = 1e-5


@pytest.fixture(scope="module")
def nmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf as m
    return m


def _start(prob, K, n_iter):
    V, D = prob.A.shape
    W0, H0 = synth.init_factors(0xF4, V, D, K)
    W, H, _ = fh.run(prob.A, W0, H0, n_iter)
    return W0, H0, f32(W), f32(H)


def _gpu_iteration(nmf, A, K, W0, H0, W, H, prec):
    import torch
    ctx = nmf.from_dense(A, K, W0=torch.from_numpy(W0).cuda(), H0=torch.from_numpy(H0).cuda(), prec=prec)
    ctx.set_factors(W, H)
    ctx.iterate(1)
    return ctx.get_factors()


@pytest.mark.parametrize("kind,K,n_iter", [("att", 80, 5), ("pie", 160, 1)])
def test_fp32_one_iteration_faces(nmf, kind, K, n_iter):
    prob = synth.faces_like(kind)
    W0, H0, W, H = _start(prob, K, n_iter)
    W64, H64 = W.astype(np.float64), H.astype(np.float64)
    dW, dH = fp32_storage_sensitivity(prob.A, W64, H64)
    assert dW < 0.3 * TOL_ITER and dH < 0.3 * TOL_ITER
    Wg, Hg = _gpu_iteration(nmf, prob.A, K, W0, H0, W, H, nmf.PREC_FP32)
    Wr, Hr = fh.iteration(prob.A, W64, H64, EPS)
    print(kind, K, "W", rel_w(Wg, Wr), "H", rel_h(Hg, Hr), "floor", dW, dH)
    assert rel_h(Hg, Hr) < TOL_ITER
    assert rel_w(Wg, Wr) < TOL_ITER


def test_bf16_one_iteration_pie(nmf):
    prob = synth.faces_like("pie")
    K = 160
    W0, H0, W, H = _start(prob, K, 1)
    W64, H64 = W.astype(np.float64), H.astype(np.float64)
    Wg, Hg = _gpu_iteration(nmf, prob.A, K, W0, H0, W, H, nmf.PREC_BF16)
    Wb, Hb = fh.iteration(prob.A, W64, H64, EPS, operand_round=round_bf16_split)
    print("pie bf16 W", rel_w(Wg, Wb), "H", rel_h(Hg, Hb))
    assert rel_w(Wg, Wb) < 2e-2 and rel_h(Hg, Hb) < 2e-2
