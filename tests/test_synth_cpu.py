"""Synthetic input generators (CPU): the face-image-shaped dense matrices
have the shapes of the paper's Table 4 (AT&T 400 x 10,304; PIE 11,554 x
4,096), pixel-like values in (0, 1] with maximum 1, and are their planted
factors' product up to the stated noise."""

import numpy as np
import pytest

from paper_1904_07935_b300 import synth


@pytest.mark.parametrize("kind,shape,r", [("att", (400, 10304), 200), ("pie", (11554, 4096), 256)])
def test_faces_like_shape_range_and_planted_factors(kind, shape, r):
    prob = synth.faces_like(kind)
    A = prob.A
    assert A.shape == shape and A.dtype == np.float32 and A.flags["C_CONTIGUOUS"]
    assert A.min() > 0.0 and A.max() == np.float32(1.0)
    assert prob.W0.shape == (shape[0], r) and prob.H0.shape == (r, shape[1])
    assert prob.W0.min() >= 0.0 and prob.H0.min() >= 0.0
    rows = np.arange(0, shape[0], max(1, shape[0] // 50))            # a sample of rows
    resid = A[rows].astype(np.float64) - prob.W0[rows] @ prob.H0
    # |N(0, 0.01^2)| noise scaled by 1 / max(A) < 1: non-negative, mean below 0.008, far below 0.05
    assert resid.min() >= -1e-6 and resid.mean() < 8e-3 and resid.max() < 0.05
    if kind == "att":                                                # deterministic
        assert np.array_equal(synth.faces_like(kind).A[:3], A[:3])
