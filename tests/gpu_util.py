"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np
import pytest

F32_EPS = 2.0 ** -24


def drgb_module():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but CUDA is not available")
    from paper_2603_04035_gb300 import build
    build.build()
    import paper_2603_04035_gb300 as drgb
    return drgb


def check_knn(X, rows, gi, gd, oi, od, k, tie_ulps=16):
    """Compare GPU k-NN rows (gi, gd) with the oracle's (oi, od) for the given rows.

    Distances must agree to FP32 accuracy position by position (they are the
    sorted k smallest, whatever the tie resolution).  Index mismatches are
    allowed only where the two candidates' FP64 squared distances differ by
    less than ``tie_ulps`` FP32 ulps of the k-th squared distance (a
    documented near-tie).  Returns the number of tie-resolved mismatches.
    """
    X64 = np.asarray(X, np.float64)
    gi = np.asarray(gi, np.int64)
    assert gi.shape == oi.shape
    # validity: distinct, in range, not self
    assert gi.min() >= 0 and gi.max() < X64.shape[0]
    assert np.all(gi != np.asarray(rows)[:, None])
    srt = np.sort(gi, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0), "duplicate neighbour in a row"
    scale = np.maximum(od[:, -1:], 1e-30)
    np.testing.assert_allclose(gd, od, rtol=4e-6, atol=4e-6 * scale.max())
    mism = gi != oi
    if mism.any():
        r, c = np.nonzero(mism)
        q = X64[np.asarray(rows)[r]]
        dg = ((X64[gi[r, c]] - q) ** 2).sum(1)
        do = ((X64[oi[r, c]] - q) ** 2).sum(1)
        tol = tie_ulps * F32_EPS * (od[r, -1] ** 2)
        assert np.all(np.abs(dg - do) <= tol), "index mismatch that is not a near-tie"
        # the set of neighbours may differ only at the k-th boundary by near-ties
        for rr in np.unique(r):
            missing = np.setdiff1d(oi[rr], gi[rr])
            qv = X64[rows[rr]]
            dm = ((X64[missing] - qv) ** 2).sum(1)
            assert np.all(dm >= (od[rr, -1] ** 2) - tie_ulps * F32_EPS * od[rr, -1] ** 2)
    return int(mism.sum())


def epoch_tolerance(ref, rtol=1e-5):
    """Per-coordinate bound |gpu - ref| <= rtol * max(|ref|, 1)."""
    return rtol * np.maximum(np.abs(ref), 1.0)
