"""Parity of the CUDA path with the oracle for the two variants of open
readings (HWENO_VARIANT_RAW_COMBINE = oracle limit_in_place 0,
HWENO_VARIANT_MEAN_EIGEN = oracle char_state 1), alone and together, in 1D
and 2D: the right-hand side within the tolerance of the default's parity
tests, and Runge-Kutta runs (relative L1 1e-12 in FP64, 1e-4 in FP32)."""

import numpy as np
import pytest

from gpu_util import (band_cells, band_cells2d, gpu_rhs1d, gpu_rhs2d, gpu_run1d, mixed_euler,
                      mixed_euler2d, rhs_tolerance, rhs_tolerance2d, round_to, square_domain)
from oracle import oracle as O
from paper_2002_08816_gb300 import hweno as H

pytestmark = pytest.mark.gpu

VARIANTS = [H.HWENO_VARIANT_RAW_COMBINE, H.HWENO_VARIANT_MEAN_EIGEN,
            H.HWENO_VARIANT_RAW_COMBINE | H.HWENO_VARIANT_MEAN_EIGEN]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _okw(variant):
    return dict(limit_in_place=0 if variant & H.HWENO_VARIANT_RAW_COMBINE else 1,
                char_state=1 if variant & H.HWENO_VARIANT_MEAN_EIGEN else 0)


@pytest.mark.parametrize("prec", [H.HWENO_FP64, H.HWENO_FP32])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx", [257, 3001])
def test_rhs1d_variant(nx, variant, prec):
    u = round_to(prec, mixed_euler(nx, nx))
    cfg = H.make_config(1, H.HWENO_EULER, nx, bc=H.HWENO_BC_OUTFLOW, precision=prec,
                        variant=variant)
    ocfg = O.Cfg1D.make(O.EULER, nx, 0.0, 1.0, O.BC_OUTFLOW, **_okw(variant))
    rg, lg, fg = gpu_rhs1d(cfg, u)
    ro, lo, fo, ind = O.rhs1d(ocfg, u)
    near, excl = band_cells(ind, ocfg.kxrcf_threshold, nx, False)
    assert np.array_equal(fg[~near], fo[~near])
    tol = rhs_tolerance(prec, ocfg, u)
    d = np.abs(rg - ro)[:, :, ~excl]
    assert d.max() <= tol, (d.max(), tol)
    # ulim_out holds the modified moments in every variant
    dl = np.abs(lg - lo)[:, :, ~excl]
    assert dl.max() <= 256 * (1e-16 if prec == H.HWENO_FP64 else 6e-8) * (np.abs(u).max() + 1)


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-4)])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("mode,nsteps", [(H.HWENO_TROUBLED_ALL, 45), (H.HWENO_TROUBLED_HYBRID, 6)])
def test_run1d_variant(mode, nsteps, variant, prec, tol):
    """Every cell troubled (no KXRCF decision), or the hybrid scheme for 6
    steps.  With unmodified first moments in the combination nothing controls
    the first moments: the hybrid run flags many cells near the threshold and
    the all-troubled run amplifies rounding (two FP64 runs part by ~10 % after
    45 steps), so that variant is compared over 5 steps (one step agrees to
    1e-15); the interface-mean variant alone over 45."""
    if variant & H.HWENO_VARIANT_RAW_COMBINE:
        nsteps = min(nsteps, 5)
    nx = 2000
    u = round_to(prec, mixed_euler(nx, 11))
    cfg = H.make_config(1, H.HWENO_EULER, nx, bc=H.HWENO_BC_OUTFLOW, cfl=0.5, precision=prec,
                        variant=variant, troubled_mode=mode)
    ocfg = O.Cfg1D.make(O.EULER, nx, 0.0, 1.0, O.BC_OUTFLOW, troubled_mode=mode, **_okw(variant))
    got, t, _ = gpu_run1d(cfg, u, nsteps)
    ref, t_o, _ = O.run1d(ocfg, u, nsteps=nsteps, cfl=0.5)
    assert np.abs(got - ref).sum() / np.abs(ref).sum() <= tol
    assert abs(t - t_o) <= (1e-13 if prec == H.HWENO_FP64 else 1e-6) * t_o


@pytest.mark.parametrize("prec", [H.HWENO_FP64, H.HWENO_FP32])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("ng", [2, 3])
def test_rhs2d_variant(ng, variant, prec):
    nx, ny = 40, 24
    dom = square_domain(nx, ny)
    u = round_to(prec, mixed_euler2d(nx, ny, dom, 7))
    cfg = H.make_config(2, H.HWENO_EULER, nx, ny, x0=dom[0], x1=dom[1], y0=dom[2], y1=dom[3],
                        bc=H.HWENO_BC_PERIODIC, lin_w=(0.96, 0.01, 0.01, 0.01, 0.01), cfl=0.4,
                        precision=prec, n_gauss=ng, variant=variant)
    ocfg = O.Cfg2D.make(O.EULER, nx, ny, *dom, O.BC_PERIODIC, n_gauss=ng, **_okw(variant))
    rg, lg, fg = gpu_rhs2d(cfg, u)
    ro, lo, fo, ind = O.rhs2d(ocfg, u)
    near, excl = band_cells2d(ind, ocfg.kxrcf_threshold, True)
    assert np.array_equal(fg[~near], fo[~near])
    assert fo.sum() > 0
    tol = rhs_tolerance2d(prec, ocfg, u)
    d = np.abs(rg - ro)[:, :, ~excl]
    assert d.max() <= tol, (d.max(), tol)


@pytest.mark.parametrize("variant", VARIANTS)
def test_run2d_variant_fp64(variant):
    nx, ny = 40, 24
    dom = square_domain(nx, ny)
    u = mixed_euler2d(nx, ny, dom, 7)
    cfg = H.make_config(2, H.HWENO_EULER, nx, ny, x0=dom[0], x1=dom[1], y0=dom[2], y1=dom[3],
                        bc=H.HWENO_BC_PERIODIC, lin_w=(0.96, 0.01, 0.01, 0.01, 0.01), cfl=0.4,
                        precision=H.HWENO_FP64, n_gauss=3, variant=variant)
    ocfg = O.Cfg2D.make(O.EULER, nx, ny, *dom, O.BC_PERIODIC, n_gauss=3, **_okw(variant))
    got, t, _ = gpu_run1d(cfg, u, 12)
    ref, t_o, _ = O.run2d(ocfg, u, nsteps=12, cfl=0.4)
    assert np.abs(got - ref).sum() / np.abs(ref).sum() <= 1e-12
    assert abs(t - t_o) <= 1e-13 * t_o


def test_adjoint_rejects_variants():
    import torch
    nx = ny = 16
    dom = square_domain(nx, ny)
    cfg = H.make_config(2, H.HWENO_EULER, nx, ny, x0=dom[0], x1=dom[1], y0=dom[2], y1=dom[3],
                        bc=H.HWENO_BC_PERIODIC, lin_w=(0.96, 0.01, 0.01, 0.01, 0.01),
                        precision=H.HWENO_FP64, variant=H.HWENO_VARIANT_MEAN_EIGEN)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        u = np.ascontiguousarray(mixed_euler2d(nx, ny, dom, 1))
        H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP64, False)
        with pytest.raises(H.HwenoError) as ei:
            H.hweno_record(h, 2, 1)
        assert ei.value.status == H.HWENO_ERR_ARG
    finally:
        H.hweno_destroy(h)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("ng", [2, 3])
def test_run2d_variant_fp32(ng, variant):
    """FP32 runs (the packed-FP32 Euler path; with the raw combination the
    stage reads an own cell's unmodified moments back from its input) over 5
    steps against the oracle, relative L1 1e-4."""
    nx, ny = 40, 24
    dom = square_domain(nx, ny)
    u = round_to(H.HWENO_FP32, mixed_euler2d(nx, ny, dom, 7))
    cfg = H.make_config(2, H.HWENO_EULER, nx, ny, x0=dom[0], x1=dom[1], y0=dom[2], y1=dom[3],
                        bc=H.HWENO_BC_PERIODIC, lin_w=(0.96, 0.01, 0.01, 0.01, 0.01), cfl=0.4,
                        precision=H.HWENO_FP32, n_gauss=ng, variant=variant)
    ocfg = O.Cfg2D.make(O.EULER, nx, ny, *dom, O.BC_PERIODIC, n_gauss=ng, **_okw(variant))
    got, t, _ = gpu_run1d(cfg, u, 5)
    ref, t_o, _ = O.run2d(ocfg, u, nsteps=5, cfl=0.4)
    assert np.abs(got - ref).sum() / np.abs(ref).sum() <= 1e-4
    assert abs(t - t_o) <= 1e-6 * t_o
