"""GPU-side test helpers: run the C ABI on torch device buffers and the oracle
on the same inputs.  Tolerances (derivation in each function) are shared by
the parity tests."""

import numpy as np

from oracle import oracle as O
from paper_2002_08816_gb300 import hweno as H
from paper_2002_08816_gb300 import workloads as W

EPS = {H.HWENO_FP64: np.finfo(np.float64).eps, H.HWENO_FP32: np.finfo(np.float32).eps}


def torch_dtype(prec):
    import torch
    return torch.float64 if prec == H.HWENO_FP64 else torch.float32


def round_to(prec, u):
    """The inputs both sides see: the state rounded to the kernel's precision."""
    return u.astype(np.float32).astype(np.float64) if prec == H.HWENO_FP32 else u.copy()


def make_pair(system, nx, x0, x1, bc, prec, mode=H.HWENO_TROUBLED_HYBRID, lin_w=None, cfl=0.5):
    lw = lin_w if lin_w is not None else (0.98, 0.01, 0.01)
    cfg = H.make_config(1, system, nx, x0=x0, x1=x1, bc=bc, lin_w=lw, cfl=cfl, precision=prec,
                        troubled_mode=mode)
    ocfg = O.Cfg1D.make(system, nx, x0, x1, bc, lin_w=lw, troubled_mode=mode)
    return cfg, ocfg


def gpu_rhs1d(cfg, u):
    import torch
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dt = torch_dtype(cfg.precision)
        uin = torch.from_numpy(np.ascontiguousarray(u)).to("cuda", dt)
        out = torch.empty_like(uin)
        ulim = torch.empty_like(uin)
        flags = torch.zeros(cfg.nx, dtype=torch.uint8, device="cuda")
        H.hweno_rhs(h, uin.data_ptr(), out.data_ptr(), flags.data_ptr(), ulim.data_ptr())
        torch.cuda.synchronize()
        return (out.double().cpu().numpy(), ulim.double().cpu().numpy(),
                flags.cpu().numpy())
    finally:
        H.hweno_destroy(h)


def gpu_run1d(cfg, u, nsteps, t_final=-1.0, chunks=1):
    import torch
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dt = torch_dtype(cfg.precision)
        uin = torch.from_numpy(np.ascontiguousarray(u)).to("cuda", dt)
        H.hweno_set_state(h, uin.data_ptr(), cfg.precision, True)
        t = None
        per = [nsteps // chunks] * chunks
        per[-1] += nsteps - sum(per)
        for k in per:
            t = H.hweno_step(h, k, t_final)
        out = torch.empty_like(uin)
        H.hweno_get_state(h, out.data_ptr(), cfg.precision, True)
        stats = H.hweno_stats(h)
        torch.cuda.synchronize()
        return out.double().cpu().numpy(), t, stats
    finally:
        H.hweno_destroy(h)


def flux_scale(ocfg, u):
    """max over cells of |f(ubar)| + alpha |ubar|: the size of the terms the
    Lax-Friedrichs flux adds."""
    a = O.alpha1d(ocfg, u)
    C = u.shape[0]
    ub = u[:, 0, :]
    if ocfg.system == O.BURGERS:
        f = 0.5 * ub[0] ** 2
        return float(np.max(np.abs(f) + a * np.abs(ub[0])))
    s = 0.0
    for i in range(0, ub.shape[1], max(1, ub.shape[1] // 4096)):
        F = O.euler1d_flux(ocfg.gas_gamma, ub[:, i])
        s = max(s, float(np.max(np.abs(F) + a * np.abs(ub[:, i]))))
    return s


def rhs_tolerance(prec, ocfg, u):
    """Absolute tolerance on L: each entry is a difference of Lax-Friedrichs
    fluxes (terms of size flux_scale) divided by dx, after a chain of a few
    dozen roundings in the kernel's precision: 256 eps * flux_scale / dx."""
    dx = (ocfg.x1 - ocfg.x0) / ocfg.nx
    return 256.0 * EPS[prec] * flux_scale(ocfg, u) / dx


def band_cells(ind, thr, nx, periodic, radius=3):
    """Cells within `radius` of a cell whose indicator lies within 1e-6
    (relative) of the threshold: there the flag may legitimately differ and
    the right-hand side with it."""
    near = np.abs(ind - thr) <= 1e-6 * max(thr, 1e-300)
    mask = np.zeros(nx, dtype=bool)
    for i in np.nonzero(near)[0]:
        for d in range(-radius, radius + 1):
            j = i + d
            if periodic:
                mask[j % nx] = True
            elif 0 <= j < nx:
                mask[j] = True
    return near, mask


# ------------------------------------------------------------------------- inputs

def mixed_burgers(nx, seed):
    """Piecewise-smooth Burgers data with two jumps (moments by Gauss)."""
    rng = np.random.default_rng(seed)
    a, b = rng.uniform(0.2, 0.45), rng.uniform(0.55, 0.85)
    amp = rng.uniform(0.3, 0.8)

    def f(x):
        return (0.5 + amp * np.sin(2 * np.pi * x) + 0.8 * (x > a) - 1.1 * (x > b))
    return W.cell_moments_1d(f, nx, 0.0, 1.0)


def mixed_euler(nx, seed):
    return W.euler_two_state_1d(nx, seed)


# ------------------------------------------------------------------------- 2D

def square_domain(nx, ny, h=None):
    """(x0, x1, y0, y1) with square cells of side h (default 1/max(nx, ny))."""
    h = h if h is not None else 1.0 / max(nx, ny)
    return 0.0, nx * h, 0.0, ny * h


def make_pair2d(system, nx, ny, dom, bc, prec, mode=H.HWENO_TROUBLED_HYBRID, ng=3, cfl=0.4,
                lin_w=None):
    lw = lin_w if lin_w is not None else (0.96, 0.01, 0.01, 0.01, 0.01)
    x0, x1, y0, y1 = dom
    cfg = H.make_config(2, system, nx, ny, x0=x0, x1=x1, y0=y0, y1=y1, bc=bc, lin_w=lw, cfl=cfl,
                        precision=prec, troubled_mode=mode, n_gauss=ng)
    ocfg = O.Cfg2D.make(system, nx, ny, x0, x1, y0, y1, bc, lin_w=lw, troubled_mode=mode,
                        n_gauss=ng)
    return cfg, ocfg


def gpu_rhs2d(cfg, u):
    import torch
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dt = torch_dtype(cfg.precision)
        uin = torch.from_numpy(np.ascontiguousarray(u)).to("cuda", dt)
        out = torch.empty_like(uin)
        ulim = torch.empty_like(uin)
        flags = torch.zeros(cfg.ny * cfg.nx, dtype=torch.uint8, device="cuda")
        H.hweno_rhs(h, uin.data_ptr(), out.data_ptr(), flags.data_ptr(), ulim.data_ptr())
        torch.cuda.synchronize()
        return (out.double().cpu().numpy(), ulim.double().cpu().numpy(),
                flags.cpu().numpy().reshape(cfg.ny, cfg.nx))
    finally:
        H.hweno_destroy(h)


gpu_run2d = gpu_run1d  # the stepping entry points do not depend on the dimension


def flux_scale2d(ocfg, u):
    ax, ay = O.alpha2d(ocfg, u)
    ub = u[:, 0]
    if ocfg.system == O.BURGERS:
        return float(np.max(0.5 * ub[0] ** 2 + max(ax, ay) * np.abs(ub[0])))
    rho, m, n, E = ub
    p = (ocfg.gas_gamma - 1) * (E - 0.5 * (m * m + n * n) / rho)
    f = np.abs(m) + np.abs(m * m / rho + p) + np.abs(m * n / rho) + np.abs(m / rho * (E + p))
    g = np.abs(n) + np.abs(m * n / rho) + np.abs(n * n / rho + p) + np.abs(n / rho * (E + p))
    return float(np.max(np.maximum(f, g) + max(ax, ay) * np.abs(ub).sum(axis=0)))


def rhs_tolerance2d(prec, ocfg, u):
    """As in 1D: 256 eps x the Lax-Friedrichs term size / dx."""
    dx = (ocfg.x1 - ocfg.x0) / ocfg.nx
    return 256.0 * EPS[prec] * flux_scale2d(ocfg, u) / dx


def band_cells2d(ind, thr, periodic, radius=3):
    near = np.abs(ind - thr) <= 1e-6 * max(thr, 1e-300)
    ny, nx = ind.shape
    mask = np.zeros_like(near)
    for j, i in zip(*np.nonzero(near)):
        for dj in range(-radius, radius + 1):
            for di in range(-radius, radius + 1):
                jj, ii = j + dj, i + di
                if periodic:
                    mask[jj % ny, ii % nx] = True
                elif 0 <= jj < ny and 0 <= ii < nx:
                    mask[jj, ii] = True
    return near, mask


def mixed_burgers2d(nx, ny, dom, seed):
    rng = np.random.default_rng(seed)
    a, b = rng.uniform(0.3, 0.7, size=2)
    x0, x1, y0, y1 = dom
    Lx, Ly = x1 - x0, y1 - y0

    def f(x, y):
        return (0.5 + 0.4 * np.sin(2 * np.pi * x / Lx) * np.cos(2 * np.pi * y / Ly)
                + 0.8 * (x > a * Lx) * (y > b * Ly))
    return W.cell_moments_2d(f, nx, ny, x0, x1, y0, y1, 3)


def mixed_euler2d(nx, ny, dom, seed):
    """Four constant quadrants plus density modes (shocks and smooth parts)."""
    rng = np.random.default_rng(seed)
    st = [(rng.uniform(0.3, 1.0), rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8),
           rng.uniform(0.3, 1.0)) for _ in range(4)]
    x0, x1, y0, y1 = dom
    xs, ys = x0 + 0.55 * (x1 - x0), y0 + 0.45 * (y1 - y0)

    def f(x, y):
        q = (x >= xs).astype(int) + 2 * (y >= ys).astype(int)
        comp = [np.choose(q, [s[k] for s in st]) for k in range(4)]
        rho = comp[0] * (1 + 0.1 * np.sin(2 * np.pi * (x - x0) / (x1 - x0) * 3)
                         * np.sin(2 * np.pi * (y - y0) / (y1 - y0) * 2))
        return W.euler_conserved_2d(rho, comp[1], comp[2], comp[3])
    return W.cell_moments_2d(f, nx, ny, x0, x1, y0, y1, 3)
