"""Parity of the CUDA 2D path (through the C ABI) with the FP64 oracle
(Sec. 2.2).  Same bars as in 1D: flags bit-exact off the threshold band, L
within gpu_util.rhs_tolerance2d, states after steps within a relative L1 of
1e-12 (FP64) or 1e-5 / 1e-4 (FP32 smooth / shocked)."""

import numpy as np
import pytest

from gpu_util import (band_cells2d, gpu_rhs2d, gpu_run2d, make_pair2d, mixed_burgers2d,
                      mixed_euler2d, rhs_tolerance2d, round_to, square_domain)
from oracle import oracle as O
from paper_2002_08816_gb300 import hweno as H
from paper_2002_08816_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = [H.HWENO_FP64, H.HWENO_FP32]
SIZES = [(4, 4), (5, 7), (16, 16), (17, 33), (40, 24)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _compare_rhs(system, nx, ny, bc, prec, mode, ng, seed, u=None, dom=None):
    dom = dom or square_domain(nx, ny)
    if u is None:
        u = (mixed_burgers2d(nx, ny, dom, seed) if system == H.HWENO_BURGERS
             else mixed_euler2d(nx, ny, dom, seed))
    u = round_to(prec, u)
    cfg, ocfg = make_pair2d(system, nx, ny, dom, bc, prec, mode, ng)
    rg, lg, fg = gpu_rhs2d(cfg, u)
    ro, lo, fo, ind = O.rhs2d(ocfg, u)
    near, excl = band_cells2d(ind, ocfg.kxrcf_threshold, bc == H.HWENO_BC_PERIODIC)
    assert np.array_equal(fg[~near], fo[~near]), "flags differ outside the threshold band"
    tol = rhs_tolerance2d(prec, ocfg, u)
    ok = ~excl
    d = np.abs(rg - ro)[:, :, ok]
    assert d.size == 0 or d.max() <= tol, (d.max(), tol)
    ltol = 256 * (1e-16 if prec == H.HWENO_FP64 else 6e-8) * (np.abs(u).max() + 1.0)
    dl = np.abs(lg - lo)[:, :, ok]
    assert dl.size == 0 or dl.max() <= ltol, (dl.max(), ltol)
    return fo


def _near_threshold_state2d(system, nx, ny, thr, seed):
    """Data constant in y (the y-jumps vanish) whose x-walk puts every cell's
    KXRCF indicator at thr (1 + delta), |delta| log-uniform in [1e-5, 0.3] on
    either side, for square cells of side 1/nx: with the left inflow face,
    jx = (u_i - 6 v_i) - (u_{i-1} + 6 v_{i-1}) = s k u_i and
    k = thr (1 + delta) h (dx + dy) / dy, h = sqrt(dx^2 + dy^2) / 2."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / nx
    k0 = thr * np.sqrt(2.0) * dx  # thr h (dx + dy) / dy with dy = dx
    delta = rng.choice([-1.0, 1.0], nx) * 10.0 ** rng.uniform(-5.0, np.log10(0.3), nx)
    sgn = rng.choice([-1.0, 1.0], nx)
    v = rng.uniform(-0.05, 0.05, nx) * dx
    w = np.empty(nx)
    w[0] = 1.0
    for i in range(1, nx):
        w[i] = (w[i - 1] + 6.0 * (v[i - 1] + v[i])) / (1.0 - sgn[i] * k0 * (1.0 + delta[i]))
    ones = np.ones((ny, 1))
    avg, mom, zero = ones * w, ones * v, np.zeros((ny, nx))
    if system == H.HWENO_BURGERS:
        return np.stack([np.stack([avg, mom, zero])])
    flat = np.full((ny, nx), 2.5)
    return np.stack([np.stack([avg, mom, zero]), np.stack([0.1 * avg, 0.1 * mom, zero]),
                     np.stack([zero, zero, zero]), np.stack([flat, zero, zero])])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("system", [H.HWENO_BURGERS, H.HWENO_EULER])
def test_flags2d_near_threshold(system, prec):
    """Most cells' indicators within 30 % of the threshold (the FP32 kernel then
    decides many with its float-pair evaluation): flags bit-exact outside the
    1e-6 band."""
    nx, ny = 512, 8
    dom = square_domain(nx, ny)
    cfg, ocfg = make_pair2d(system, nx, ny, dom, H.HWENO_BC_PERIODIC, prec,
                            H.HWENO_TROUBLED_HYBRID, 2)
    u = round_to(prec, _near_threshold_state2d(system, nx, ny, ocfg.kxrcf_threshold,
                                               seed=3 + system))
    _, _, fo, ind = O.rhs2d(ocfg, u)
    rel = np.abs(ind / ocfg.kxrcf_threshold - 1.0)
    assert ((rel > 1e-6) & (rel < 0.3)).sum() > 0.8 * rel.size
    assert 0.2 < fo.mean() < 0.8
    _compare_rhs(system, nx, ny, H.HWENO_BC_PERIODIC, prec, H.HWENO_TROUBLED_HYBRID, 2, seed=0,
                 u=u, dom=dom)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [H.HWENO_BC_PERIODIC, H.HWENO_BC_OUTFLOW])
@pytest.mark.parametrize("size", SIZES)
@pytest.mark.parametrize("system", [H.HWENO_BURGERS, H.HWENO_EULER])
def test_rhs2d(system, size, bc, prec):
    _compare_rhs(system, size[0], size[1], bc, prec, H.HWENO_TROUBLED_HYBRID, 3, seed=size[0])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("system", [H.HWENO_BURGERS, H.HWENO_EULER])
@pytest.mark.parametrize("mode", [H.HWENO_TROUBLED_ALL, H.HWENO_TROUBLED_NONE])
@pytest.mark.parametrize("ng", [2, 3])
def test_rhs2d_modes_and_quadrature(mode, system, prec, ng):
    _compare_rhs(system, 20, 18, H.HWENO_BC_PERIODIC, prec, mode, ng, seed=4)


@pytest.mark.parametrize("ng", [2, 3])
def test_rhs2d_two_point_gauss_hybrid(ng):
    fl = _compare_rhs(H.HWENO_EULER, 33, 21, H.HWENO_BC_OUTFLOW, H.HWENO_FP64,
                      H.HWENO_TROUBLED_HYBRID, ng, seed=7)
    assert 0 < fl.sum() < 0.6 * fl.size


def _compare_run(system, nx, ny, bc, prec, nsteps, u, dom, tol, ng=3, cfl=0.4, t_final=-1.0):
    u = round_to(prec, u)
    cfg, ocfg = make_pair2d(system, nx, ny, dom, bc, prec, H.HWENO_TROUBLED_HYBRID, ng, cfl)
    got, tg, st = gpu_run2d(cfg, u, nsteps, t_final)
    ref, to, nt = O.run2d(ocfg, u, nsteps=nsteps, cfl=cfl, t_final=t_final)
    rel = np.abs(got - ref).sum() / np.abs(ref).sum()
    assert rel <= tol, (rel, tol)
    assert abs(tg - to) <= (1e-13 if prec == H.HWENO_FP64 else 1e-6) * max(to, 1e-30)
    return st, nt


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-5)])
def test_run2d_smooth_density_wave(prec, tol):
    n = 24
    _compare_run(H.HWENO_EULER, n, n, H.HWENO_BC_PERIODIC, prec, 6,
                 W.euler_density_wave_2d(n, n), (0.0, 2.0, 0.0, 2.0), tol)


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-4)])
def test_run2d_shocked_quadrants(prec, tol):
    nx, ny = 36, 28
    dom = square_domain(nx, ny)
    st, nt = _compare_run(H.HWENO_EULER, nx, ny, H.HWENO_BC_OUTFLOW, prec, 5,
                          mixed_euler2d(nx, ny, dom, 12), dom, tol)
    assert nt > 0


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-4)])
def test_run2d_burgers_to_final_time(prec, tol):
    n = 32
    dom = (0.0, 4.0, 0.0, 4.0)
    _compare_run(H.HWENO_BURGERS, n, n, H.HWENO_BC_PERIODIC, prec, 50,
                 W.burgers_sine_2d(n, n), dom, tol, cfl=0.5, t_final=0.5 / np.pi)


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-11), (H.HWENO_FP32, 1e-4)])
def test_run2d_burgers_shock_example_3_9(prec, tol):
    """Example 3.9: Example 3.3's data through the shock to T = 1.5/pi with the
    paper's CFL 0.6 (the oracle's run is pinned against the entropy solution)."""
    n = 40
    dom = (0.0, 4.0, 0.0, 4.0)
    st, nt = _compare_run(H.HWENO_BURGERS, n, n, H.HWENO_BC_PERIODIC, prec, 200,
                          W.burgers_sine_2d(n, n), dom, tol, cfl=0.6, t_final=1.5 / np.pi)
    assert nt > 0 and st["troubled"] > 0


def test_periodic_conservation_2d_fp64():
    n = 24
    dom = square_domain(n, n)
    u = mixed_euler2d(n, n, dom, 3)
    cfg, _ = make_pair2d(H.HWENO_EULER, n, n, dom, H.HWENO_BC_PERIODIC, H.HWENO_FP64)
    got, _, _ = gpu_run2d(cfg, u, 10)
    np.testing.assert_allclose(got[:, 0].sum(axis=(1, 2)), u[:, 0].sum(axis=(1, 2)), rtol=1e-12)


@pytest.mark.parametrize("ng", [2, 3])
def test_full_size_vortex_modes_fp32_sampled(ng):
    """The 4096 x 4096 vortex-plus-modes 2D Euler workload in FP32 (the launch
    configuration of the 2D measurement): L on the whole grid from the GPU,
    checked on sampled 7 x 7 windows against the oracle evaluated on those
    windows with the global alpha_x, alpha_y (a 7-cell margin keeps the
    window's own boundary out of the compared cells)."""
    import torch  # noqa: F401
    n = 4096
    u = W.euler_vortex_modes_2d(n, n, seed=2026, npts=2).astype(np.float32).astype(np.float64)
    cfg, ocfg = make_pair2d(H.HWENO_EULER, n, n, (0.0, 10.0, 0.0, 10.0), H.HWENO_BC_PERIODIC,
                            H.HWENO_FP32, ng=ng)
    rg, _, fg = gpu_rhs2d(cfg, u)
    ax, ay = O.alpha2d(ocfg, u)
    rng = np.random.default_rng(5)
    m = 7
    h = 10.0 / n
    for _ in range(12):
        j0, i0 = rng.integers(0, n, size=2)
        js = np.arange(j0 - m - 3, j0 + m + 4) % n
        is_ = np.arange(i0 - m - 3, i0 + m + 4) % n
        win = u[:, :, js][:, :, :, is_]
        nw = win.shape[-1]
        wcfg = O.Cfg2D.make(O.EULER, nw, nw, 0.0, nw * h, 0.0, nw * h, O.BC_OUTFLOW,
                            lin_w=tuple(cfg.lin_w), n_gauss=ng)
        ro, _, fo, ind = O.rhs2d(wcfg, win, ax, ay)
        c = slice(m, m + 7)
        sub_g = rg[:, :, js[c]][:, :, :, is_[c]]
        sub_o = ro[:, :, c, c]
        tol = rhs_tolerance2d(H.HWENO_FP32, wcfg, win)
        assert np.max(np.abs(sub_g - sub_o)) <= tol
        near = np.abs(ind[c, c] - 1.0) <= 1e-6
        assert np.array_equal(fg[js[c]][:, is_[c]][~near], fo[c, c][~near])
