"""Fixed-W H subproblem, FP64 — test infrastructure.

With W fixed, the H half of Alg. 1 (R <- A^T W, S <- W^T W, then the k loop)
is one sweep of exact coordinate descent on the strictly convex problem
    min_{h >= eps} 1/2 ||a - W h||^2
for every document column a, provided S_kk = 1 (W with unit columns, as the
normalisation step of Alg. 1 leaves it).  Repeating the sweep converges to the
unique NNLS optimum h*.  This module runs those sweeps to convergence and also
provides two independent exact solvers used to pin them:
* ``nnls_lawson_hanson`` — scipy.optimize.nnls (Lawson & Hanson, 1974);
* ``nnls_bruteforce`` — enumerate all passive sets (K <= 10), keep the one
  that satisfies the KKT conditions.
"""

from __future__ import annotations

import itertools

import numpy as np

from .fast_hals import update_h


def hals_sweeps(Rt: np.ndarray, S: np.ndarray, H0: np.ndarray, eps: float,
                tol: float = 1e-12, max_sweeps: int = 100000):
    """Repeat the H loop of Alg. 1 with fixed R (D x K) and S until the
    largest change of any entry is below ``tol``.  Returns (H, sweeps)."""
    H = np.array(H0, dtype=np.float64)
    for it in range(1, max_sweeps + 1):
        Hn = update_h(Rt, S, H, eps)
        delta = float(np.max(np.abs(Hn - H))) if H.size else 0.0
        H = Hn
        if delta < tol:
            return H, it
    return H, max_sweeps


def nnls_lawson_hanson(W: np.ndarray, a: np.ndarray) -> np.ndarray:
    from scipy.optimize import nnls
    x, _ = nnls(np.asarray(W, dtype=np.float64), np.asarray(a, dtype=np.float64))
    return x


def nnls_bruteforce(W: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Exact NNLS by enumerating passive sets (only for K <= 10)."""
    W = np.asarray(W, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    K = W.shape[1]
    if K > 10:
        raise ValueError("brute force is for K <= 10")
    best, best_f = None, np.inf
    for r in range(K + 1):
        for Pset in itertools.combinations(range(K), r):
            x = np.zeros(K)
            if Pset:
                idx = list(Pset)
                sol, *_ = np.linalg.lstsq(W[:, idx], a, rcond=None)
                if np.any(sol < 0):
                    continue
                x[idx] = sol
            g = W.T @ (W @ x - a)            # gradient of 1/2||a - Wx||^2
            zero = [k for k in range(K) if k not in Pset]
            if zero and np.any(g[zero] < -1e-10):
                continue
            f = 0.5 * float(np.sum((a - W @ x) ** 2))
            if f < best_f:
                best, best_f = x, f
    return best
