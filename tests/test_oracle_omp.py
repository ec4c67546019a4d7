"""The oracle's OpenMP build (per-cell loops of Eq. (odeH) and Eq. (ode2)
spread over threads, the arithmetic unchanged) gives bitwise the results of
the plain build, so the all-core CPU baseline times the same computation."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2002_08816_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _omp():
    if O.lib_omp() is None:
        pytest.skip("gcc has no OpenMP here")
    O.threads(4)


def test_omp_1d_bitwise():
    nx = 3000
    u = W.euler_riemann_1d(nx, (1.0, 0.75, 1.0), (0.125, 0.0, 0.1), 0.0, 1.0, 0.5)
    cfg = O.Cfg1D.make(O.EULER, nx, 0.0, 1.0, O.BC_REFLECTIVE)
    a, ta, na = O.run1d(cfg, u, nsteps=40, cfl=0.5)
    b, tb, nb = O.run1d(cfg, u, nsteps=40, cfl=0.5, omp=True)
    assert na > 0 and na == nb and ta == tb
    assert np.array_equal(a, b)


def test_omp_2d_bitwise():
    n = 40
    u = W.euler_quadrants_2d(n, n, seed=3, npts=3)
    cfg = O.Cfg2D.make(O.EULER, n, n, 0.0, 10.0, 0.0, 10.0, O.BC_PERIODIC, n_gauss=2)
    a, ta, na = O.run2d(cfg, u, nsteps=4, cfl=0.5)
    b, tb, nb = O.run2d(cfg, u, nsteps=4, cfl=0.5, omp=True)
    assert na > 0 and na == nb and ta == tb
    assert np.array_equal(a, b)
