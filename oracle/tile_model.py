"""Data-movement model of Sec. 3.2 (Eq. 3) and Sec. 5 (Eqs. 7-11).

Test infrastructure; pinned by the numbers the paper prints in Sec. 5.  C is
the cache size in words (8-byte FP64 words), V, D, K, T as in the paper.
"""

from __future__ import annotations

import math


def fast_hals_total(V: float, D: float, K: float, C: float) -> float:
    """Eq. 3: total words moved by one iteration of Alg. 1."""
    rc = 1.0 / math.sqrt(C)
    return K * (K * (V + D) * (1 + 2 * rc) + 4 * V * D * rc + 6 * V + 3 * D + 2 * K + 1)


def fast_hals_w_loop(V: float, K: float) -> float:
    """Sec. 3.2: words moved by the W loop of Alg. 1, K(VK + K + 6V + 1)."""
    return K * (V * K + K + 6 * V + 1)


def phase13_volume(V: float, K: float, T: float, C: float) -> float:
    """Eq. 7 (closed form on its right-hand side)."""
    return V * T * T * (1.0 / T + 2.0 / math.sqrt(C)) * (K * K - K * T) / (2 * T * T)


def phase2_volume(V: float, K: float, T: float) -> float:
    """Eq. 8: (K/T) T (VT + T + V)."""
    return (K / T) * T * (V * T + T + V)


def vol(V: float, K: float, T: float, C: float) -> float:
    """Eq. 9: V(1/T + 2/sqrt(C))(K^2 - KT) + (K/T) T (V T)."""
    return V * (1.0 / T + 2.0 / math.sqrt(C)) * (K * K - K * T) + (K / T) * T * (V * T)


def tile_size_printed(K: float, C: float) -> float:
    """Eq. 11 as printed: T = sqrt(K - 2/sqrt(C))."""
    return math.sqrt(K - 2.0 / math.sqrt(C))


def tile_size_stationary(K: float, C: float) -> float:
    """Stationary point of Eq. 9 in T (d vol / dT = 0, solved exactly).

    d/dT [V K^2/T + 2VK^2/sqrt(C) - VK - 2VKT/sqrt(C) + V K T]
      = -V K^2 / T^2 + V K (1 - 2/sqrt(C)) = 0  =>  T = sqrt(K / (1 - 2/sqrt(C))).
    Eq. 10 as printed has T^2 (2/sqrt(C) - 1) + K = 0, whose root is the same
    value; Eq. 11 drops the division.  Both are close to sqrt(K).
    """
    return math.sqrt(K / (1.0 - 2.0 / math.sqrt(C)))


CACHE_35MB_WORDS = 35 * 2 ** 20 / 8
