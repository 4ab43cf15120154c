import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libdigs.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


# A (pixel, Gaussian) pair whose squared Mahalanobis distance E lies within FP32 rounding of the cutoff
# (relative margin ~1e-7) is decided by rounding: the kernels' float32 evaluation may include it where the
# float64 oracle does not.  Such a pair changes that Gaussian's gradient at the 1e-3 level (one boundary
# pixel), so element-by-element gradient tests leave Gaussians with a margin below this out.
CUTOFF_AMBIGUOUS = 2e-6


def unambiguous(wl, w_rows, views, delta=CUTOFF_AMBIGUOUS):
    """Indices of the Gaussians of workload `wl` none of whose pairs in `views` (weights w_rows) lies
    within `delta` (relative) of the cutoff, by the oracle's float64 E."""
    import numpy as np
    from oracle import digs_oracle as O
    m = O.cutoff_margin(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), wl.lattice, wl.phi, w_rows,
                        views)
    return np.nonzero(m > delta)[0]
