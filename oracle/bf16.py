"""BF16 rounding, written from the format's definition — test infrastructure.

bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits of
an IEEE binary32 value.  Rounding to nearest, ties to even, of a binary32
pattern u: add 0x7FFF plus the lowest kept bit ((u >> 16) & 1), then clear
the low 16 bits.  (NaN/Inf do not occur in the factorisation's operands.)

The split form carries a binary32 value x as the pair hi = bf16(x),
lo = bf16(x - hi); x - hi is exact in binary32 (both are multiples of x's
binary32 ulp and the difference is at most half a bf16 ulp of x), so the pair
represents x to within 2^-16 |x|.
"""

import numpy as np


def round_bf16(x) -> np.ndarray:
    """Nearest bfloat16 value (ties to even) of float32(x), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_bf16_split(x) -> np.ndarray:
    """Value carried by the BF16 pair (hi, lo) of float32(x): hi + lo with
    hi = bf16(x) and lo = bf16(x - hi), returned as float64."""
    f = np.asarray(np.asarray(x, dtype=np.float32), dtype=np.float64)
    hi = round_bf16(f)
    lo = round_bf16(f - hi)          # f - hi is exact (see the module note)
    return hi + lo
