"""Shared test helpers: running the oracle and the GPU library on one scene,
and the parity measures used by the GPU tests."""
import numpy as np


def state_rel_err(Ra, Ta, Xa, Rb, Tb, Xb):
    """max |a - b| / max(|b|, s) with s = 1 m for positions and points and 1
    for rotation-matrix entries (which are bounded by 1)."""
    e = 0.0
    e = max(e, float(np.max(np.abs(np.asarray(Ra) - np.asarray(Rb)))))
    for a, b in ((Ta, Tb), (Xa, Xb)):
        a, b = np.asarray(a), np.asarray(b)
        if a.size:
            e = max(e, float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))))
    return e


def rms_inliers(err, outlier):
    return float(np.sqrt(np.mean(np.asarray(err)[~np.asarray(outlier)] ** 2)))
