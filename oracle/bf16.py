"""BF16 rounding, written from the format's definition — test infrastructure.

bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits of
an IEEE binary32 value.  Rounding to nearest, ties to even, of a binary32
pattern u: add 0x7FFF plus the lowest kept bit ((u >> 16) & 1), then clear
the low 16 bits.  (NaN/Inf do not occur in the factorisation's operands.)
"""

import numpy as np


def round_bf16(x) -> np.ndarray:
    """Nearest bfloat16 value (ties to even) of float32(x), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
