"""Multiplicative updates (Lee & Seung, "Algorithms for non-negative matrix
factorization", NIPS 2001) in FP64 — test infrastructure for the MU
comparator (the paper names MU as the simplest NMF algorithm, Sec. 2, and
compares PL-NMF with it, Sec. 6).

The paper gives no formula; the standard Frobenius-norm rules are used:
    H <- H * (W^T A) / (W^T W H + delta)
    W <- W * (A H^T) / (W H H^T + delta)
elementwise, H first (with the current W), then W (with the new H).
Readings: delta = 1e-16 (the same small constant as the HALS eps) keeps a
zero denominator from producing 0/0; W is not normalised (the objective is
invariant to the scaling W D, D^-1 H).  The objective ||A - W H||_F^2 does
not increase under either rule (Lee & Seung 2001, Theorem 1).
"""

from __future__ import annotations

import numpy as np

from .fast_hals import DEFAULT_EPS, _as_operator, normalize_init

DEFAULT_DELTA = DEFAULT_EPS


def update_h(A, W: np.ndarray, H: np.ndarray, delta: float = DEFAULT_DELTA) -> np.ndarray:
    """H <- H * (W^T A) / (W^T W H + delta); A is V x D (dense or sparse)."""
    Aop = _as_operator(A)
    W = np.asarray(W, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    num = np.asarray((Aop.T @ W).T)                   # W^T A, K x D
    den = (W.T @ W) @ H + delta
    return H * num / den


def update_w(A, W: np.ndarray, H: np.ndarray, delta: float = DEFAULT_DELTA) -> np.ndarray:
    """W <- W * (A H^T) / (W H H^T + delta)."""
    Aop = _as_operator(A)
    W = np.asarray(W, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    num = np.asarray(Aop @ H.T)                       # A H^T, V x K
    den = W @ (H @ H.T) + delta
    return W * num / den


def iteration(A, W: np.ndarray, H: np.ndarray, delta: float = DEFAULT_DELTA):
    """One MU iteration: H with the current W, then W with the new H."""
    H = update_h(A, W, H, delta)
    W = update_w(A, W, H, delta)
    return W, H


def run(A, W0: np.ndarray, H0: np.ndarray, n_iter: int, delta: float = DEFAULT_DELTA, normalize: bool = True):
    """MU for a fixed number of iterations from (W0, H0); W0's columns are
    scaled to unit norm first (the same start the HALS runs use)."""
    W = normalize_init(W0) if normalize else np.array(W0, dtype=np.float64)
    H = np.array(H0, dtype=np.float64)
    for _ in range(n_iter):
        W, H = iteration(A, W, H, delta)
    return W, H
