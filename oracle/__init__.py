"""FP64 CPU oracle for the FAST-HALS / PL-NMF iteration — TEST INFRASTRUCTURE.

This package is the checker, not the product.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the CUDA library never calls it and shares no code with it.  Inputs come
from :mod:`paper_1904_07935_b300.synth` (which holds no method arithmetic).

Modules
-------
fast_hals   Alg. 1 of the paper, literally (un-reordered), FP64.
pl_nmf      Alg. 2 (three-phase tiled reorder) in FP64, used to pin the
            reorder identity stated in Sec. 3.3.
objective   Eq. 2 directly and through the trace identity; the relative
            objective of Sec. 6.2.2.
nnls        Fixed-W H subproblem (the H half of Alg. 1 repeated to
            convergence) and exact NNLS references for pins.
mlp         FP64 forward / backward / Adam of the warm-start network.
bf16        round-to-nearest-even to bfloat16 (operands of the BF16 form).
tile_model  Data-movement model, Eq. 3 and Eqs. 7-11 (Sec. 5).

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` against closed forms, library routines, brute
force or the paper's printed numbers; none is "parity unpinned".
"""
