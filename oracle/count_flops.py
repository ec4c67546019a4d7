"""Algorithmic flops per cell-stage, counted on the oracle (test and
measurement infrastructure; writes oracle/flop_counts.json, which bench.py
reads for the arithmetic rooflines).

  python oracle/count_flops.py

One evaluation of the right-hand side of Eq. (odeH) (1D) or Eq. (ode2) (2D)
by the op-counting build of the oracle (the oracle's C sources compiled with a
scalar that counts its operations: opcount.cpp) on periodic grids of N and
2N cells, with every cell smooth (troubled mode NONE: the linear p0 path) and
with every cell troubled (mode ALL: the limiter and the characteristic HWENO
path); the difference over N is the cost of one cell (the count is affine in
N: a few hundred operations per call do not depend on the grid), and the
Runge-Kutta combination of Eq. (RK) (2 flops per value: one multiply-add) is
added.  Operations counted one flop each: add/sub, mul,
div, sqrt and pow (pow appears only where a smoothness indicator squares a
sum); comparisons, fabs and copies are free.  The evaluation includes what
the oracle does per stage besides the reconstruction: the wave speeds of
alpha, the KXRCF indicator and the limiter's inputs.
"""

import ctypes
import json
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(_HERE))

from oracle import oracle as O  # noqa: E402
from paper_2002_08816_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(_HERE, "flop_counts.json")
NX1, NX2 = 256, 64


def ops1d(system, mode, nx):
    """[add/sub, mul, div, sqrt, pow] of one 1D evaluation on nx cells"""
    cfg = O.Cfg1D.make(system, nx, 0.0, 1.0, O.BC_PERIODIC, troubled_mode=mode)
    u = W.euler_two_state_1d(nx, seed=3) if system == O.EULER else W.burgers_sine_1d(nx)
    u = np.ascontiguousarray(u.reshape(-1), dtype=np.float64)
    rhs, ulim = np.empty_like(u), np.empty_like(u)
    fl, ind = np.zeros(nx, np.uint8), np.zeros(nx)

    def call(L):
        st = L.hwo1d_rhs(ctypes.byref(cfg), O._p(u), -1.0, O._p(rhs), O._p(ulim),
                         fl.ctypes.data_as(O._PU8), O._p(ind))
        assert st == 0
    return O.count_ops(call)


def ops2d(system, mode, ng, nx, ny):
    """the same for one 2D evaluation on nx x ny square cells"""
    cfg = O.Cfg2D.make(system, nx, ny, 0.0, 10.0, 0.0, 10.0 * ny / nx, O.BC_PERIODIC,
                       troubled_mode=mode, n_gauss=ng)
    if system == O.EULER:
        u = W.euler_vortex_modes_2d(nx, ny, seed=2026, npts=2)
    else:
        u = W.burgers_sine_2d(nx, ny)
    u = np.ascontiguousarray(u.reshape(-1), dtype=np.float64)
    rhs, ulim = np.empty_like(u), np.empty_like(u)
    fl, ind = np.zeros(nx * ny, np.uint8), np.zeros(nx * ny)

    def call(L):
        st = L.hwo2d_rhs(ctypes.byref(cfg), O._p(u), -1.0, -1.0, O._p(rhs), O._p(ulim),
                         fl.ctypes.data_as(O._PU8), O._p(ind))
        assert st == 0
    return O.count_ops(call)


def _count1d(system, mode):
    a, b = ops1d(system, mode, NX1), ops1d(system, mode, 2 * NX1)
    return [y - x for x, y in zip(a, b)], NX1, 2 * (3 if system == O.EULER else 1)


def _count2d(system, mode, ng):
    a, b = ops2d(system, mode, ng, NX2, NX2), ops2d(system, mode, ng, NX2, 2 * NX2)
    return [y - x for x, y in zip(a, b)], NX2 * NX2, 3 * (4 if system == O.EULER else 1)


def table():
    """{path: {"ops": [add/sub, mul, div, sqrt, pow] per cell, "rhs": flops
    per cell of one evaluation of L, "cell_stage": rhs + the RK combination}}"""
    cases = {}
    for sysname, system in (("euler", O.EULER), ("burgers", O.BURGERS)):
        for path, mode in (("smooth", O.TROUBLED_NONE), ("troubled", O.TROUBLED_ALL)):
            cases["1d_%s_%s" % (sysname, path)] = _count1d(system, mode)
            for ng in (2, 3):
                cases["2d_%s_ng%d_%s" % (sysname, ng, path)] = _count2d(system, mode, ng)
    out = {}
    for name, (ops, ncell, values) in cases.items():
        per = [v / ncell for v in ops]
        rhs = sum(per)
        out[name] = {"ops": per, "rhs": rhs, "cell_stage": rhs + 2 * values}
    return out


def main():
    t = table()
    with open(OUT, "w") as f:
        json.dump({"note": "oracle op counts per cell-stage (oracle/count_flops.py)", "paths": t},
                  f, indent=1, sort_keys=True)
    for k in sorted(t):
        print("%-26s %9.1f flops per cell-stage" % (k, t[k]["cell_stage"]))


if __name__ == "__main__":
    main()
