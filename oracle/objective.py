"""Objective of Eq. 2 and the relative objective of Sec. 6.2.2, FP64.

Test infrastructure.  Two independent evaluations:

* ``frob2_direct``: sum over all entries of (A - WH)^2, formed entry by entry
  (dense), or for sparse A as the sum over stored entries of (a - (WH))^2 plus
  the sum over absent entries of (WH)^2, with WH formed in row blocks.
* ``frob2_trace``: the expansion ||A||^2 - 2<W, A H^T> + <W^T W, H H^T>.

The relative objective is sqrt(frob2 / ||A||_F^2) (Sec. 6.2.2).
"""

from __future__ import annotations

import numpy as np

from .fast_hals import _as_operator


def _is_sparse(M) -> bool:
    import scipy.sparse as sp
    return sp.issparse(M)


def norm2_A(A) -> float:
    Aop = _as_operator(A)
    if _is_sparse(Aop):
        return float(np.sum(Aop.data.astype(np.float64) ** 2))
    return float(np.sum(Aop * Aop))


def frob2_direct(A, W, H, block_rows: int = 2048) -> float:
    """sum_{v,d} (A_vd - (WH)_vd)^2, accumulated in FP64."""
    W = np.asarray(W, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    Aop = _as_operator(A)
    V = W.shape[0]
    total = 0.0
    for r0 in range(0, V, block_rows):
        r1 = min(V, r0 + block_rows)
        WH = W[r0:r1] @ H
        if _is_sparse(Aop):
            Ab = Aop[r0:r1].toarray()
        else:
            Ab = Aop[r0:r1]
        Rb = Ab - WH
        total += float(np.sum(Rb * Rb))
    return total


def frob2_trace(A, W, H) -> float:
    """||A||^2 - 2 <W, A H^T> + <W^T W, H H^T>, all in FP64."""
    W = np.asarray(W, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    Aop = _as_operator(A)
    P = np.asarray(Aop @ H.T)
    return norm2_A(A) - 2.0 * float(np.sum(W * P)) + float(np.sum((W.T @ W) * (H @ H.T)))


def relative_error(A, W, H, direct: bool = False) -> float:
    """sqrt(sum (A - WH)^2 / sum A^2) (Sec. 6.2.2)."""
    f = frob2_direct(A, W, H) if direct else frob2_trace(A, W, H)
    return float(np.sqrt(max(f, 0.0) / norm2_A(A)))
