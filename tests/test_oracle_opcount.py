"""The op-counting build of the oracle (oracle/opcount.cpp: the oracle's C
sources compiled as C++ with a counting scalar), which gives the algorithmic
flops of the arithmetic rooflines: its results are bitwise those of the plain
build (the counting scalar performs each operation once, in the source's
order, as an IEEE double operation), its counts scale with the grid, the
square roots are the ones the formulas have, and the stored table
(oracle/flop_counts.json, read by bench.py) is current."""

import ctypes
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2002_08816_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


def _rhs1d(L, cfg, u):
    u = np.ascontiguousarray(u.reshape(-1), dtype=np.float64)
    rhs, ulim = np.empty_like(u), np.empty_like(u)
    fl, ind = np.zeros(cfg.nx, np.uint8), np.zeros(cfg.nx)
    assert L.hwo1d_rhs(ctypes.byref(cfg), O._p(u), -1.0, O._p(rhs), O._p(ulim),
                       fl.ctypes.data_as(O._PU8), O._p(ind)) == 0
    return rhs, ulim, fl


def _rhs2d(L, cfg, u):
    u = np.ascontiguousarray(u.reshape(-1), dtype=np.float64)
    rhs, ulim = np.empty_like(u), np.empty_like(u)
    fl, ind = np.zeros(cfg.nx * cfg.ny, np.uint8), np.zeros(cfg.nx * cfg.ny)
    assert L.hwo2d_rhs(ctypes.byref(cfg), O._p(u), -1.0, -1.0, O._p(rhs), O._p(ulim),
                       fl.ctypes.data_as(O._PU8), O._p(ind)) == 0
    return rhs, ulim, fl


@pytest.mark.parametrize("mode", [O.TROUBLED_HYBRID, O.TROUBLED_NONE, O.TROUBLED_ALL])
def test_counting_build_is_bitwise_the_plain_build(mode):
    nx = 300
    for system, u in ((O.EULER, W.euler_two_state_1d(nx, seed=5)),
                      (O.BURGERS, W.burgers_sine_1d(nx))):
        cfg = O.Cfg1D.make(system, nx, 0.0, 1.0, O.BC_OUTFLOW, troubled_mode=mode)
        a = _rhs1d(O.lib(), cfg, u)
        b = _rhs1d(O.lib_opcount(), cfg, u)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    n = 24
    for ng in (2, 3):
        cfg = O.Cfg2D.make(O.EULER, n, n, 0.0, 10.0, 0.0, 10.0, O.BC_PERIODIC,
                           troubled_mode=mode, n_gauss=ng)
        u = W.euler_quadrants_2d(n, n, seed=7)
        a = _rhs2d(O.lib(), cfg, u)
        b = _rhs2d(O.lib_opcount(), cfg, u)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_counts_are_affine_in_the_grid_and_match_the_formulas():
    from oracle.count_flops import ops1d, ops2d
    for system in (O.EULER, O.BURGERS):
        for mode in (O.TROUBLED_NONE, O.TROUBLED_ALL):
            a, b, c = (np.array(ops1d(system, mode, n)) for n in (256, 512, 768))
            assert np.array_equal(c - b, b - a), (system, mode, a, b, c)
    a, b, c = (np.array(ops2d(O.EULER, O.TROUBLED_NONE, 2, 16, n)) for n in (16, 32, 48))
    assert np.array_equal(c - b, b - a)
    # smooth cells: Euler's one square root per cell is the sound speed of its
    # wave speed (alpha); Burgers has none
    e = np.array(ops1d(O.EULER, O.TROUBLED_NONE, 512)) - np.array(ops1d(O.EULER, O.TROUBLED_NONE, 256))
    assert e[3] == 256
    bg = np.array(ops1d(O.BURGERS, O.TROUBLED_NONE, 512)) - np.array(ops1d(O.BURGERS, O.TROUBLED_NONE, 256))
    assert bg[3] == 0
    # the troubled path costs several times the smooth one (limiter and HWENO)
    t = np.array(ops1d(O.EULER, O.TROUBLED_ALL, 512)) - np.array(ops1d(O.EULER, O.TROUBLED_ALL, 256))
    assert t.sum() > 4 * e.sum()


def test_stored_table_is_current():
    from oracle import count_flops
    path = os.path.join(os.path.dirname(O.__file__), "flop_counts.json")
    stored = json.load(open(path))["paths"]
    fresh = count_flops.table()
    assert set(stored) == set(fresh)
    for k in fresh:
        assert abs(stored[k]["cell_stage"] - fresh[k]["cell_stage"]) <= 1e-9 * fresh[k]["cell_stage"], k
