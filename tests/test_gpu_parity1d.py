"""Parity of the CUDA 1D path (through the C ABI) with the FP64 oracle.

Flags: bit-exact outside the 1e-6 band around the KXRCF threshold.  Right-hand
sides: elementwise within gpu_util.rhs_tolerance.  States after Runge-Kutta
steps: relative L1 within 1e-12 in FP64; in FP32 within 1e-5 on smooth data
and 1e-4 on shocked data (the accuracy targets of the FP32 path).
"""

import numpy as np
import pytest

from gpu_util import (band_cells, gpu_rhs1d, gpu_run1d, make_pair, mixed_burgers, mixed_euler,
                      rhs_tolerance, round_to)
from oracle import oracle as O
from paper_2002_08816_gb300 import hweno as H
from paper_2002_08816_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = [H.HWENO_FP64, H.HWENO_FP32]
SIZES = [4, 5, 37, 256, 257, 1000, 3001]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _compare_rhs(system, nx, bc, prec, mode, seed, u=None, x0=0.0, x1=1.0):
    if u is None:
        u = mixed_burgers(nx, seed) if system == H.HWENO_BURGERS else mixed_euler(nx, seed)
    u = round_to(prec, u)
    cfg, ocfg = make_pair(system, nx, x0, x1, bc, prec, mode)
    rhs_g, lim_g, fl_g = gpu_rhs1d(cfg, u)
    rhs_o, lim_o, fl_o, ind = O.rhs1d(ocfg, u)
    near, excl = band_cells(ind, ocfg.kxrcf_threshold, nx, bc == H.HWENO_BC_PERIODIC)
    keep = ~near
    assert np.array_equal(fl_g[keep], fl_o[keep]), "flags differ outside the threshold band"
    tol = rhs_tolerance(prec, ocfg, u)
    ok = ~excl
    diff = np.abs(rhs_g - rhs_o)[:, :, ok]
    assert diff.size == 0 or diff.max() <= tol, (diff.max(), tol)
    ltol = 256 * (1e-16 if prec == H.HWENO_FP64 else 6e-8) * (np.abs(u).max() + 1.0)
    dl = np.abs(lim_g - lim_o)[:, :, ok]
    assert dl.size == 0 or dl.max() <= ltol, (dl.max(), ltol)
    return fl_o


def _near_threshold_walk(nx, thr, h, seed):
    """Cell averages built cell by cell so that the KXRCF indicator of every
    cell (left inflow face: u >= 0) is thr (1 + delta), |delta| log-uniform in
    [1e-5, 0.3] on either side: the zone where an FP32 evaluation alone cannot
    decide the flag, yet outside the 1e-6 band where the flag may differ.  The
    jump (u_i - 6 v_i) - (u_{i-1} + 6 v_{i-1}) = s k u_i, k = thr h (1 + delta),
    fixes u_i from u_{i-1} and the moments."""
    rng = np.random.default_rng(seed)
    delta = rng.choice([-1.0, 1.0], nx) * 10.0 ** rng.uniform(-5.0, np.log10(0.3), nx)
    sgn = rng.choice([-1.0, 1.0], nx)
    v = rng.uniform(-0.05, 0.05, nx) * h
    u = np.empty(nx)
    u[0] = 1.0
    for i in range(1, nx):
        k = thr * h * (1.0 + delta[i])
        u[i] = (u[i - 1] + 6.0 * (v[i - 1] + v[i])) / (1.0 - sgn[i] * k)
    return u, v


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["burgers", "euler-rho", "euler-E"])
def test_flags_near_threshold(prec, case):
    """Most cells' indicators within 30 % of the threshold (the FP32 kernel
    then decides with its error-free float-pair evaluation, the FP64 kernel
    as the oracle does): flags bit-exact outside the 1e-6 band."""
    nx = 4096
    system = H.HWENO_BURGERS if case == "burgers" else H.HWENO_EULER
    cfg, ocfg = make_pair(system, nx, 0.0, 1.0, H.HWENO_BC_OUTFLOW, prec)
    thr, h = ocfg.kxrcf_threshold, 0.5 / nx
    w, v = _near_threshold_walk(nx, thr, h, seed=len(case) + 7 * prec)
    if system == H.HWENO_BURGERS:
        u = np.stack([w, v])[None]
    else:
        flat, zero = np.full(nx, 2.5), np.zeros(nx)
        rho, vr, E, vE = (w, v, flat, zero) if case == "euler-rho" else (flat, zero, w, v)
        u = np.stack([np.stack([rho, vr]), np.stack([0.1 * rho, 0.1 * vr]), np.stack([E, vE])])
    u = round_to(prec, u)
    _, _, fl_o, ind = O.rhs1d(ocfg, u)
    rel = np.abs(ind / thr - 1.0)
    zone = (rel > 1e-6) & (rel < 0.3)
    assert zone.sum() > 0.8 * nx, zone.sum()
    assert 0.2 * nx < fl_o.sum() < 0.8 * nx
    _compare_rhs(system, nx, H.HWENO_BC_OUTFLOW, prec, H.HWENO_TROUBLED_HYBRID, seed=0, u=u)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [H.HWENO_BC_PERIODIC, H.HWENO_BC_OUTFLOW])
@pytest.mark.parametrize("nx", SIZES)
def test_rhs_burgers(prec, bc, nx):
    _compare_rhs(H.HWENO_BURGERS, nx, bc, prec, H.HWENO_TROUBLED_HYBRID, seed=nx)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [H.HWENO_BC_PERIODIC, H.HWENO_BC_OUTFLOW, H.HWENO_BC_REFLECTIVE])
@pytest.mark.parametrize("nx", SIZES)
def test_rhs_euler(prec, bc, nx):
    _compare_rhs(H.HWENO_EULER, nx, bc, prec, H.HWENO_TROUBLED_HYBRID, seed=nx)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("system", [H.HWENO_BURGERS, H.HWENO_EULER])
@pytest.mark.parametrize("mode", [H.HWENO_TROUBLED_ALL, H.HWENO_TROUBLED_NONE])
def test_rhs_all_and_none_modes(prec, system, mode):
    _compare_rhs(system, 700, H.HWENO_BC_PERIODIC, prec, mode, seed=5)


def test_rhs_has_troubled_and_smooth_cells():
    """The mixed inputs exercise both branches of the hybrid switch."""
    fl = _compare_rhs(H.HWENO_EULER, 3001, H.HWENO_BC_OUTFLOW, H.HWENO_FP64,
                      H.HWENO_TROUBLED_HYBRID, seed=3001)
    assert 0 < fl.sum() < 0.5 * fl.size


@pytest.mark.parametrize("prec", PRECS)
def test_rhs_full_size_euler_two_state(prec):
    """At the 65536-cell 1D Euler workload the oracle still evaluates L in well
    under a second, so all outputs are compared."""
    _compare_rhs(H.HWENO_EULER, 65536, H.HWENO_BC_OUTFLOW, prec, H.HWENO_TROUBLED_HYBRID,
                 seed=20250)


def _compare_run(system, nx, bc, prec, nsteps, u, x0, x1, tol, cfl=0.5, t_final=-1.0,
                 mode=H.HWENO_TROUBLED_HYBRID, chunks=1):
    u = round_to(prec, u)
    cfg, ocfg = make_pair(system, nx, x0, x1, bc, prec, mode, cfl=cfl)
    got, t_g, stats = gpu_run1d(cfg, u, nsteps, t_final, chunks)
    ref, t_o, nt = O.run1d(ocfg, u, nsteps=nsteps, cfl=cfl, t_final=t_final)
    rel = np.abs(got - ref).sum() / np.abs(ref).sum()
    assert rel <= tol, (rel, tol)
    assert abs(t_g - t_o) <= (1e-13 if prec == H.HWENO_FP64 else 1e-6) * max(t_o, 1e-30)
    return stats, nt


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-5)])
def test_run_burgers_smooth(prec, tol):
    """Example 3.1 data, 40 steps: no troubled cell."""
    nx = 400
    stats, nt = _compare_run(H.HWENO_BURGERS, nx, H.HWENO_BC_PERIODIC, prec, 40,
                             W.burgers_sine_1d(nx), -1.0, 1.0, tol)
    assert nt == 0 and stats["troubled"] == 0


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-4)])
def test_run_burgers_shock_to_final_time(prec, tol):
    """Example 3.5 at N = 400 (the FP64 Burgers workload): run to T = 1.5/pi
    with CFL 0.6, clipped final step, through the shock."""
    nx = 400
    stats, nt = _compare_run(H.HWENO_BURGERS, nx, H.HWENO_BC_PERIODIC, prec, 400,
                             W.burgers_sine_1d(nx), -1.0, 1.0, tol, cfl=0.6,
                             t_final=1.5 / np.pi, chunks=3)
    assert nt > 0
    assert stats["troubled"] == nt if prec == H.HWENO_FP64 else stats["troubled"] > 0


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-4)])
def test_run_euler_two_state(prec, tol):
    """Seeded two-state 1D Euler data with outflow ends, 45 steps (crosses the
    32-step graph and the single-step graph)."""
    nx = 2000
    _compare_run(H.HWENO_EULER, nx, H.HWENO_BC_OUTFLOW, prec, 45, mixed_euler(nx, 11), 0.0, 1.0,
                 tol)


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-5)])
def test_run_euler_smooth_density_wave(prec, tol):
    nx = 320
    _compare_run(H.HWENO_EULER, nx, H.HWENO_BC_PERIODIC, prec, 60, W.euler_density_wave_1d(nx),
                 0.0, 2.0, tol)


def test_run_full_size_euler_fp32():
    """65536-cell two-state Euler workload, FP32, the launch configuration the
    benchmark times, 8 steps against the oracle."""
    nx = 65536
    _compare_run(H.HWENO_EULER, nx, H.HWENO_BC_OUTFLOW, H.HWENO_FP32, 8,
                 W.euler_two_state_1d(nx, seed=20250), 0.0, 1.0, 1e-4)


def test_periodic_conservation_fp64():
    import torch  # noqa: F401
    nx = 1024
    u = mixed_burgers(nx, 2)
    cfg, _ = make_pair(H.HWENO_BURGERS, nx, 0.0, 1.0, H.HWENO_BC_PERIODIC, H.HWENO_FP64)
    got, _, _ = gpu_run1d(cfg, u, 50)
    assert abs(got[0, 0].sum() - u[0, 0].sum()) <= 1e-12 * np.abs(u[0, 0]).sum()


def test_state_roundtrip_bit_exact():
    import torch
    nx = 777
    u = mixed_euler(nx, 4)
    for prec in PRECS:
        cfg, _ = make_pair(H.HWENO_EULER, nx, 0.0, 1.0, H.HWENO_BC_OUTFLOW, prec)
        h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
        try:
            host = np.ascontiguousarray(u, dtype=np.float64 if prec == H.HWENO_FP64 else np.float32)
            H.hweno_set_state(h, host.ctypes.data, prec, False)
            back = np.empty_like(host)
            H.hweno_get_state(h, back.ctypes.data, prec, False)
            assert np.array_equal(back, host)
            back64 = np.empty(host.shape, dtype=np.float64)
            H.hweno_get_state(h, back64.ctypes.data, H.HWENO_FP64, False)
            assert np.array_equal(back64, host.astype(np.float64))
        finally:
            H.hweno_destroy(h)


def test_nonphysical_state_is_reported():
    """A negative density reaches the status word and the step returns
    HWENO_ERR_NONPHYSICAL (no device fault, no trap)."""
    import torch
    nx = 64
    u = mixed_euler(nx, 1)
    u[0, 0, 10] = -1.0
    cfg, _ = make_pair(H.HWENO_EULER, nx, 0.0, 1.0, H.HWENO_BC_OUTFLOW, H.HWENO_FP64)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        host = np.ascontiguousarray(u)
        H.hweno_set_state(h, host.ctypes.data, H.HWENO_FP64, False)
        with pytest.raises(H.HwenoError) as ei:
            H.hweno_step(h, 2)
        assert ei.value.status == H.HWENO_ERR_NONPHYSICAL
    finally:
        H.hweno_destroy(h)


def test_step_before_set_state_is_an_error():
    import torch
    cfg, _ = make_pair(H.HWENO_BURGERS, 64, 0.0, 1.0, H.HWENO_BC_PERIODIC, H.HWENO_FP64)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(H.HwenoError) as ei:
            H.hweno_step(h, 1)
        assert ei.value.status == H.HWENO_ERR_STATE
    finally:
        H.hweno_destroy(h)


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-4)])
def test_run_blast_waves_between_walls(prec, tol):
    """Example 3.8's data (two blast waves, reflective walls), 800 cells, 40 steps."""
    nx = 800

    def g(x):
        p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
        return W.euler_conserved_1d(np.ones_like(x), np.zeros_like(x), p)
    u = W.cell_moments_1d(g, nx, 0.0, 1.0)
    stats, nt = _compare_run(H.HWENO_EULER, nx, H.HWENO_BC_REFLECTIVE, prec, 40, u, 0.0, 1.0, tol,
                             cfl=0.6)
    assert nt > 0


@pytest.mark.parametrize("system", [H.HWENO_BURGERS, H.HWENO_EULER])
def test_fp32_time_step_is_fp64(system):
    """The FP32 path's global CFL reduction and dt are FP64 (Sec. 2.1, alpha =
    max |f'(u)|; Sec. 3, CFL): after one step t equals the recorded dt, which
    is the correctly rounded FP64 quotient CFL dx / alpha of an alpha that is
    the FP64 maximum of FP32 wave speeds (so alpha is a float).  It agrees with
    the oracle's dt on the same input to the FP32 wave speeds' few ulp."""
    nx, cfl = 3001, 0.5
    u = round_to(H.HWENO_FP32, mixed_euler(nx, 9) if system == H.HWENO_EULER
                 else mixed_burgers(nx, 9))
    cfg, ocfg = make_pair(system, nx, 0.0, 1.0, H.HWENO_BC_OUTFLOW, H.HWENO_FP32, cfl=cfl)
    _, t, stats = gpu_run1d(cfg, u, 1)
    dt = stats["dt"]
    assert t == dt
    cdx = cfl * (1.0 / nx)
    alpha = np.float32(cdx / dt)
    assert cdx / np.float64(alpha) == dt
    dt_o = O.dt1d(ocfg, u, cfl)
    assert abs(dt - dt_o) <= 1e-6 * dt_o
