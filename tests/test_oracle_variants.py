"""Pins of the oracle's two variants of readings the paper leaves open:
char_state = 1 (Euler HWENO interface values in the characteristic fields of
the mean of the two averages at each interface, instead of the cell average)
and limit_in_place = 0 (the Runge-Kutta combination uses the unmodified first
moments).  Each reduces to the default where it cannot act; the interface-mean
variant keeps the fifth order; limit_in_place = 0 is the Runge-Kutta
combination of the operator's own outputs with the raw stage inputs.  The
last test reports how much each changes the 1D shock tests."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2002_08816_gb300 import workloads as W


def _mixed_euler(nx, seed):
    return W.euler_two_state_1d(nx, seed)


def test_mean_eigen_is_a_no_op_for_burgers():
    u = W.burgers_sine_1d(64)
    a = O.rhs1d(O.Cfg1D.make(O.BURGERS, 64, -1, 1, O.BC_PERIODIC, troubled_mode=O.TROUBLED_ALL), u)
    b = O.rhs1d(O.Cfg1D.make(O.BURGERS, 64, -1, 1, O.BC_PERIODIC, troubled_mode=O.TROUBLED_ALL,
                             char_state=1), u)
    assert np.array_equal(a[0], b[0])
    u2 = W.burgers_sine_2d(12, 12)
    c = O.rhs2d(O.Cfg2D.make(O.BURGERS, 12, 12, 0, 4, 0, 4, O.BC_PERIODIC,
                             troubled_mode=O.TROUBLED_ALL), u2)
    d = O.rhs2d(O.Cfg2D.make(O.BURGERS, 12, 12, 0, 4, 0, 4, O.BC_PERIODIC,
                             troubled_mode=O.TROUBLED_ALL, char_state=1), u2)
    assert np.array_equal(c[0], d[0])


def test_variants_are_no_ops_without_troubled_cells():
    u = _mixed_euler(300, 3)
    base = dict(troubled_mode=O.TROUBLED_NONE)
    ref, _, _ = O.run1d(O.Cfg1D.make(O.EULER, 300, 0, 1, O.BC_OUTFLOW, **base), u, nsteps=10, cfl=0.4)
    for kw in (dict(char_state=1), dict(limit_in_place=0)):
        got, _, _ = O.run1d(O.Cfg1D.make(O.EULER, 300, 0, 1, O.BC_OUTFLOW, **base, **kw), u,
                            nsteps=10, cfl=0.4)
        assert np.array_equal(got, ref), kw
    u2 = W.euler_quadrants_2d(14, 14, seed=5)
    c = O.rhs2d(O.Cfg2D.make(O.EULER, 14, 14, 0, 10, 0, 10, O.BC_PERIODIC, **base), u2)
    d = O.rhs2d(O.Cfg2D.make(O.EULER, 14, 14, 0, 10, 0, 10, O.BC_PERIODIC, char_state=1, **base), u2)
    assert np.array_equal(c[0], d[0])


def test_mean_eigen_uses_the_interface_mean():
    """Where the two averages at an interface are equal, their mean is that
    average, so the interface value equals the default's exactly; elsewhere
    the variant differs."""
    nx = 40
    u = _mixed_euler(nx, 9)
    u[:, :, 10:14] = u[:, :, 10:11]          # cells 10..13 identical
    cfg0 = O.Cfg1D.make(O.EULER, nx, 0, 1, O.BC_OUTFLOW, troubled_mode=O.TROUBLED_ALL)
    cfg1 = O.Cfg1D.make(O.EULER, nx, 0, 1, O.BC_OUTFLOW, troubled_mode=O.TROUBLED_ALL, char_state=1)
    f0 = O.rhs1d(cfg0, u, faces=True)[4]
    f1 = O.rhs1d(cfg1, u, faces=True)[4]
    # u^+_{i-1/2} of cells 11..13 (left neighbour equal), u^-_{i+1/2} of cells 10..12
    assert np.array_equal(f0[:, 0, 11:14], f1[:, 0, 11:14])
    assert np.array_equal(f0[:, 1, 10:13], f1[:, 1, 10:13])
    assert np.abs(f0 - f1).max() > 1e-6


def test_mean_eigen_keeps_fifth_order():
    """Example 3.2 with every cell troubled, interface-mean fields: the errors
    stay within a factor 3 of Table 2's new-HWENO column and the order >= 4.5."""
    T = 2.0
    errs = {}
    for nx in (40, 80):
        dx = 2.0 / nx
        dt = 0.6 * dx ** (5.0 / 3.0)
        ns = int(np.ceil(T / dt)) + 1
        cfg = O.Cfg1D.make(O.EULER, nx, 0.0, 2.0, O.BC_PERIODIC, troubled_mode=O.TROUBLED_ALL,
                           char_state=1)
        u, t, _ = O.run1d(cfg, W.euler_density_wave_1d(nx), nsteps=ns, t_final=T, dt_fixed=dt)
        ex = W.cell_moments_1d(lambda x: 1 + 0.2 * np.sin(np.pi * (x - T)), nx, 0, 2, 8)[0, 0]
        errs[nx] = np.mean(np.abs(u[0, 0] - ex))
    assert {40: 9.09e-07, 80: 7.89e-09}[40] / 3 < errs[40] < 3 * 9.09e-07, errs
    assert np.log(errs[40] / errs[80]) / np.log(2) > 4.5, errs


@pytest.mark.parametrize("lip", [1, 0])
def test_step_is_the_rk_combination_of_the_operator(lip):
    """One step of Eq. (RK) equals its combination written from the operator's
    outputs: with limit_in_place = 1 the stage inputs carry the modified first
    moments (ulim), with 0 the raw ones."""
    nx = 500
    u = _mixed_euler(nx, 4)
    cfg = O.Cfg1D.make(O.EULER, nx, 0, 1, O.BC_OUTFLOW, limit_in_place=lip)
    dt = 0.4 * (1.0 / nx) / O.alpha1d(cfg, u)
    got, nt = O.step1d(cfg, u, dt)
    assert nt > 0

    def stage(x):
        L, ulim, _, _ = O.rhs1d(cfg, x)
        return L, (ulim if lip else x)

    L, b0 = stage(u)
    u1 = b0 + dt * L
    L, b1 = stage(u1)
    u2 = 0.75 * b0 + 0.25 * b1 + 0.25 * dt * L
    L, b2 = stage(u2)
    u3 = (1.0 / 3.0) * b0 + (2.0 / 3.0) * b2 + (2.0 / 3.0) * dt * L
    np.testing.assert_allclose(got, u3, rtol=1e-14, atol=1e-14)


def _run_to(cfg, u, T):
    t, steps, troubled = 0.0, 0, 0
    while t < T:
        u, t, nt = O.run1d(cfg, u, nsteps=1, cfl=0.6, t0=t, t_final=T)
        steps += 1
        troubled += nt
    return u, troubled / (3.0 * cfg.nx * steps)


@pytest.mark.parametrize("name", ["lax", "shu-osher", "blast"])
def test_variants_on_the_shock_suite(name):
    """How much each variant changes Examples 3.6-3.8.  Interface-mean fields:
    the density moves by under 0.5 % (L1, relative) and the troubled share by
    under a tenth.  Unmodified first moments in the combination: the density
    moves by a few per cent, but the troubled share grows more than five-fold
    (47 / 61 / 95 % against 6.1 / 2.6 / 5.8 %; the paper prints 13.41 / 3.54 /
    13.94 %): the oscillating first moments are flagged again and again.  This
    is the evidence for storing the modified moments (the default reading)."""
    from test_oracle1d_pins import _shock_problem
    nx, x0, x1, bc, T, _, u0 = _shock_problem(name)
    ref, share0 = _run_to(O.Cfg1D.make(O.EULER, nx, x0, x1, bc), u0, T)
    out = {}
    for tag, kw in (("mean_eigen", dict(char_state=1)), ("raw_combine", dict(limit_in_place=0))):
        u, share = _run_to(O.Cfg1D.make(O.EULER, nx, x0, x1, bc, **kw), u0, T)
        rel = np.abs(u[0, 0] - ref[0, 0]).sum() / np.abs(ref[0, 0]).sum()
        out[tag] = (rel, share)
        assert np.all(u[0, 0] > 0)
    assert 0.0 < out["mean_eigen"][0] < 5e-3 and abs(out["mean_eigen"][1] - share0) < share0 / 10
    assert 0.0 < out["raw_combine"][0] < 0.1 and out["raw_combine"][1] > 5 * share0
    print(name, "default troubled share %.4f" % share0,
          {k: ("rho L1 diff %.2e" % v[0], "share %.4f" % v[1]) for k, v in out.items()})
