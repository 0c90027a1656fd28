import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def exact_4x4():
    """A 4^3 x 4 oracle path (stout-smeared seeded field, N_v = 4, full dilution) and its exact
    LapH propagator G = V^dag K^{-1} gamma_4 V from the dense LU, shared by the oracle pins.
    Tests that change the path's dilution put it back."""
    import synth
    from oracle.pipeline import OraclePath
    wl = synth.Workload(name="t", ns=4, nt=4, xi=3.5, csw=1.0, m0=-0.05, nv=4, gauge_seed=31, n_stout4d=3,
                        n_stout3d=2, dil_time=(1, 0), dil_spin=(1, 0), dil_laph=(1, 0), source_times=(0,),
                        n_noise=2)
    path = OraclePath(wl)
    return path, path.exact_G()


@pytest.fixture(scope="session")
def free_shell_6():
    """The lowest 21 eigenvectors of the free Laplacian on one 6^3 slice: eigenvalues 21 and 22
    are 4 sin^2(pi/6) = 1 and 2, so they span the plane waves of {0, +-e_x, +-e_y, +-e_z}."""
    import numpy as np
    from oracle import laplacian
    u = np.broadcast_to(np.eye(3, dtype=complex), (1, 6, 6, 6, 4, 3, 3)).copy()
    evals, v = laplacian.lowest_eigpairs(u, 22)
    assert abs(evals[0, 20] - 1.0) < 1e-10 and abs(evals[0, 21] - 2.0) < 1e-10
    return v[:, :21]
