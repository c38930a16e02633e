"""PL-NMF three-phase tiled factor update, Alg. 2 (Sec. 3.3, Eqs. 4-6), FP64.

Test infrastructure: it exists to pin the reorder identity — the paper states
that the tiled form performs exactly the same operations as Alg. 1 in a
different order (Sec. 3.3), so in FP64 it must agree with ``fast_hals`` to
rounding.

The update of one "tall" factor X (N x K) with Gram G (K x K) and data term
B (N x K) is written once and used for both factors:

    W:  X = W,   G = Q, B = P, init X_new = X_old * diag(G), normalise columns
    H:  X = H^T, G = S, B = R, init X_new = X_old,           no normalisation
        (Sec. 4.1, last sentence: H is updated "in the same fashion ... except
        for the normalization"; the init differs because the H update of Alg. 1
        has no H_k S_kk term to cancel.)

Phase 1 (Eq. 4): for every tile tau, columns left of tau get the old values
of tile tau times the matching block of G.
Phase 2 (Eq. 5, Alg. 2 inner loop): inside tile tau, column t adds B, subtracts
new columns of the tile before t and old columns from t on, clamps at eps,
and (W only) divides by its L2 norm.
Phase 3 (Eq. 6): columns right of tau get the new values of tile tau times the
matching block of G.

gamma = ceil(K / T); the last tile may be short (reading of gamma = K/T when T
does not divide K).
"""

from __future__ import annotations

import math

import numpy as np


def tiled_update(X_old: np.ndarray, G: np.ndarray, B: np.ndarray, T: int, eps: float,
                 scale_init_by_diag: bool, normalize: bool) -> np.ndarray:
    X_old = np.asarray(X_old, dtype=np.float64)
    N, K = X_old.shape
    gamma = math.ceil(K / T)
    tiles = [(tau * T, min((tau + 1) * T, K)) for tau in range(gamma)]

    # Initialise X_new from X_old (Alg. 2, loop before phase 1).
    if scale_init_by_diag:
        X_new = X_old * np.diag(G)[None, :]
    else:
        X_new = X_old.copy()

    # Phase 1: old tile tau into every column left of the tile (Eq. 4).
    for lo, hi in tiles:
        if lo > 0:
            X_new[:, :lo] -= X_old[:, lo:hi] @ G[lo:hi, :lo]

    for lo, hi in tiles:
        # Phase 2: sequential inside the tile (Eq. 5).  G[t, k] as printed;
        # G is symmetric.
        for t in range(lo, hi):
            s = X_new[:, lo:t] @ G[t, lo:t] + X_old[:, t:hi] @ G[t, t:hi]
            X_new[:, t] = np.maximum(eps, X_new[:, t] + B[:, t] - s)
            if normalize:
                X_new[:, t] /= math.sqrt(float(np.sum(X_new[:, t] * X_new[:, t])))
        # Phase 3: new tile tau into every column right of the tile (Eq. 6).
        if hi < K:
            X_new[:, hi:] -= X_new[:, lo:hi] @ G[lo:hi, hi:]
    return X_new


def update_w(P, Q, W_old, T: int, eps: float) -> np.ndarray:
    """Alg. 2: W_new from W_old, P = A H^T, Q = H H^T with tile width T."""
    return tiled_update(W_old, Q, P, T, eps, scale_init_by_diag=True, normalize=True)


def update_h(R, S, H_old, T: int, eps: float) -> np.ndarray:
    """H update in the same tiled fashion; H_old is K x D, returns K x D."""
    Ht = tiled_update(np.asarray(H_old).T, S, R, T, eps, scale_init_by_diag=False,
                      normalize=False)
    return Ht.T.copy()
