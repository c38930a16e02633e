"""B300-native FAST-HALS / PL-NMF hot path.

Importing the package loads nothing native; the CUDA library is loaded on
first use of :mod:`paper_1904_07935_b300.nmf`, and that import fails loudly
when the compiled library is missing.
"""

__all__ = ["synth", "nmf"]
