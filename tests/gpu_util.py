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
