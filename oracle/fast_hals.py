"""FAST-HALS, Alg. 1 of the paper (Sec. 3.1), in FP64 — test infrastructure.

Follows the algorithm's steps in its order and notation:
    R <- A^T W ;  S <- W^T W
    for k = 0..K-1:  H_k <- max(eps, H_k + R_k - H^T S_k)
    P <- A H^T ;  Q <- H H^T
    for k = 0..K-1:  W_k <- max(eps, W_k Q_kk + P_k - W Q_k) ;  W_k <- W_k / ||W_k||_2
H_k is row k of H (K x D) and W_k column k of W (V x K).  Both loops update
in place, so rows/columns j < k are already new when k is updated (the
sequential dependence stated in Sec. 3.3).

Readings where the paper is silent (also listed in the design notes):
* eps is not given; default 1e-16.
* W's columns are scaled to unit L2 norm at initialisation (``normalize_init``)
  so that S_kk = 1 at the first H update, which the update of H_k (no division
  by S_kk) assumes.
* "UNTIL convergence" has no criterion; callers run a fixed iteration count.
"""

from __future__ import annotations

import numpy as np

DEFAULT_EPS = 1e-16


def _as_operator(A):
    """Dense ndarray or scipy sparse matrix -> float64 object supporting @."""
    if hasattr(A, "to_scipy"):          # synth.CsrMatrix
        A = A.to_scipy()
    if hasattr(A, "tocsr"):
        return A.astype(np.float64).tocsr()
    return np.asarray(A, dtype=np.float64)


def normalize_init(W: np.ndarray) -> np.ndarray:
    """Scale every column of the initial W to unit L2 norm (reading of the
    initialisation step of Alg. 1; H is left as drawn)."""
    W = np.array(W, dtype=np.float64)
    W /= np.linalg.norm(W, axis=0, keepdims=True)
    return W


def update_h(R: np.ndarray, S: np.ndarray, H: np.ndarray, eps: float = DEFAULT_EPS) -> np.ndarray:
    """Alg. 1, H loop: for k ascending, H_k <- max(eps, H_k + R_k - H^T S_k).

    R is D x K (= A^T W), S is K x K (= W^T W), H is K x D.  Returns the new H
    (a copy, updated row by row in place).
    """
    H = np.array(H, dtype=np.float64)
    K = H.shape[0]
    for k in range(K):
        # H^T S_k uses the current H: rows < k are already updated.
        H[k, :] = np.maximum(eps, H[k, :] + R[:, k] - H.T @ S[:, k])
    return H


def update_w(P: np.ndarray, Q: np.ndarray, W: np.ndarray, eps: float = DEFAULT_EPS) -> np.ndarray:
    """Alg. 1, W loop: for k ascending,
    W_k <- max(eps, W_k Q_kk + P_k - W Q_k), then W_k <- W_k / ||W_k||_2.

    P is V x K (= A H^T), Q is K x K (= H H^T), W is V x K.
    """
    W = np.array(W, dtype=np.float64)
    K = W.shape[1]
    for k in range(K):
        # W Q_k uses the current W: columns < k are already new and normalised.
        W[:, k] = np.maximum(eps, W[:, k] * Q[k, k] + P[:, k] - W @ Q[:, k])
        W[:, k] = W[:, k] / np.linalg.norm(W[:, k])
    return W


def iteration(A, W: np.ndarray, H: np.ndarray, eps: float = DEFAULT_EPS, trace: dict | None = None,
              operand_round=None, a_round=None):
    """One REPEAT body of Alg. 1: update H, then W.  Returns (W, H).

    If ``trace`` is a dict it receives the intermediates R, S, H, P, Q, W.
    ``operand_round`` (e.g. bf16.round_bf16) rounds the operands of the four
    matrix products (R, S, P, Q) before they are multiplied exactly
    (FP64): the definition of a reduced-precision-product form of Alg. 1.
    ``a_round``, if given, is used for A instead (e.g. bf16.round_bf16_split,
    A carried as a BF16 pair).  The k loops stay FP64.
    """
    Aop = _as_operator(A)
    W = np.asarray(W, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    rnd = operand_round if operand_round is not None else (lambda x: x)
    if a_round is not None:
        Ar = a_round(Aop)
    else:
        Ar = Aop if operand_round is None else rnd(Aop)
    # Updating H
    Wr = rnd(W)
    R = np.asarray(Ar.T @ Wr)
    S = Wr.T @ Wr
    H = update_h(R, S, H, eps)
    # Updating W
    Hr = rnd(H)
    P = np.asarray(Ar @ Hr.T)
    Q = Hr @ Hr.T
    W = update_w(P, Q, W, eps)
    if trace is not None:
        trace.update(R=R, S=S, H=H, P=P, Q=Q, W=W)
    return W, H


def run(A, W0: np.ndarray, H0: np.ndarray, n_iter: int, eps: float = DEFAULT_EPS,
        normalize: bool = True, objective_every: int = 0, operand_round=None, a_round=None):
    """Alg. 1 for a fixed number of iterations from (W0, H0).

    Returns (W, H, history) where history lists the relative objective
    (Sec. 6.2.2) after every ``objective_every`` iterations (empty if 0).
    """
    from . import objective as obj

    W = normalize_init(W0) if normalize else np.array(W0, dtype=np.float64)
    H = np.array(H0, dtype=np.float64)
    hist = []
    for it in range(n_iter):
        W, H = iteration(A, W, H, eps, operand_round=operand_round, a_round=a_round)
        if objective_every and (it + 1) % objective_every == 0:
            hist.append(obj.relative_error(A, W, H))
    return W, H, hist
