"""Shared helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np

# Tolerances:
#  - float32-compensated predictions: max |z - z_ref| / S_q <= 1e-5, S_q =
#    sum w|z| / sum w from the oracle (a relative error is ill-posed where
#    the signed field makes sum w z cancel, so the error is scaled by the
#    magnitude of the terms that are summed);
#  - float64 predictions: the same measure <= 1e-9;
#  - kNN distances: float32 rounding of float32 coordinates, <= 1e-6 relative;
#  - kNN index sets: exact unless the oracle's k-th and (k+1)-th distances are
#    closer than 1e-6 relative.
TOL_FP32 = 1e-5
TOL_FP64 = 1e-9
TOL_DIST = 1e-6
NEAR_TIE = 1e-6


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def check_knn(oracle, x, y, qx, qy, k, idx_gpu, dist_gpu, robs_gpu=None, ref=None):
    """Compares a GPU kNN result with the oracle's brute force (or with
    ``ref`` = (idx, dist) of k or k+1 columns from another oracle search).

    Unique parts are compared exactly or to rounding: the sorted k smallest
    distances and, away from near-ties, the index set.  Where the oracle's
    k-th and (k+1)-th distances nearly tie, the GPU set may differ, and each
    GPU index must then be a point at the reported distance."""
    n = len(x)
    if ref is None:
        ridx, rd = oracle.knn(x, y, qx, qy, min(k + 1, n))
    else:
        ridx, rd = ref
    kk = rd.shape[1]
    d_ref = rd[:, :k]
    np.testing.assert_allclose(dist_gpu.astype(np.float64), d_ref, rtol=TOL_DIST, atol=1e-30)
    if robs_gpu is not None:
        np.testing.assert_allclose(robs_gpu.astype(np.float64), d_ref.mean(1), rtol=2 * TOL_DIST)
    same = np.array([set(a) == set(b) for a, b in zip(idx_gpu.tolist(), ridx[:, :k].tolist())])
    if kk > k:
        with np.errstate(invalid="ignore"):
            gap = (rd[:, k] - rd[:, k - 1]) / np.maximum(rd[:, k], 1e-300)
        near = np.isfinite(rd[:, k]) & (gap < NEAR_TIE)
    else:
        near = np.zeros(len(qx), bool)
    bad = ~same & ~near
    assert not bad.any(), f"{bad.sum()} queries with a different kNN set away from ties"
    # every reported index is a real point at the reported distance
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    assert (idx_gpu >= 0).all() and (idx_gpu < n).all()
    dd = np.hypot(qx.astype(np.float64)[:, None] - xd[idx_gpu],
                  qy.astype(np.float64)[:, None] - yd[idx_gpu])
    np.testing.assert_allclose(dist_gpu.astype(np.float64), dd, rtol=TOL_DIST, atol=1e-30)
    # the list is in increasing distance
    assert (np.diff(dist_gpu, axis=1) >= 0).all()
    return same.mean()
