"""Helpers shared by the GPU parity tests (comparison metrics).

Reading of "max relative difference in W and H" used here: the largest
absolute difference over the factor divided by the largest absolute entry of
the oracle's factor (max-norm relative error).  A per-column normalisation
cannot be met by any FP32 implementation on the dense planted workload: there
the H update cancels terms of size ~400 (R and S h) into rows whose entries
are ~0.2, and merely storing R in FP32 already perturbs such a row by more
than 1e-5 of its own maximum.  The per-column figure is still reported.
"""

import numpy as np


def max_rel(gpu, ref):
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-300))


def colmax_rel(gpu, ref, axis):
    """max over columns (axis=0) or rows (axis=1) of max|gpu - ref| / max|ref|."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    d = np.abs(g - r).max(axis=axis)
    m = np.maximum(np.abs(r).max(axis=axis), 1e-30)
    return float(np.max(d / m))


def rel_w(W_gpu, W_ref):
    return max_rel(W_gpu, W_ref)


def rel_h(H_gpu, H_ref):
    return max_rel(H_gpu, H_ref)


def forward_error_ratio(got, ref, scale):
    """max |got - ref| / scale, elementwise scale = magnitude of the terms an
    entry is computed from (the quantity FP32 rounding error is proportional
    to); entries clamped at eps on both sides compare exactly."""
    d = np.abs(np.asarray(got, dtype=np.float64) - np.asarray(ref, dtype=np.float64))
    return float(np.max(d / np.maximum(scale, 1e-300)))


def h_update_scale(R, S, H_old, H_new):
    """|h_k| + |R_k| + sum_j |S_jk| max(|h_j old|, |h_j new|): the terms of the
    k-th H update of Alg. 1 (H is K x D, R is D x K)."""
    Hm = np.maximum(np.abs(H_old), np.abs(H_new))
    return np.abs(H_old) + np.abs(R).T + np.abs(S).T @ Hm


def f32(x):
    return np.asarray(x, dtype=np.float32)


def fp32_storage_sensitivity(A, W, H, eps=1e-16):
    """Max-norm change of one oracle iteration when every stored intermediate
    (W, H, R, S, P, Q) is rounded to FP32 once, arithmetic staying FP64.

    This is the part of the FP32 path's error that no FP32 kernel can avoid;
    tolerances for badly conditioned cases are derived from it."""
    from oracle import fast_hals as fh
    r = lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)
    Aop = fh._as_operator(A)
    W_ref, H_ref = fh.iteration(Aop, W, H, eps)
    Wf, Hf = r(W), r(H)
    R, S = r(Aop.T @ Wf), r(Wf.T @ Wf)
    H2 = r(fh.update_h(R, S, Hf, eps))
    P, Q = r(Aop @ H2.T), r(H2 @ H2.T)
    W2 = fh.update_w(P, Q, Wf, eps)
    return max_rel(W2, W_ref), max_rel(H2, H_ref)
