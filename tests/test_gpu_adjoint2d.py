"""The CUDA adjoint of the 2D scheme (through the C ABI) against the oracle's
reference gradient (PyTorch autograd through the oracle's frozen-switch
stage, oracle/adjoint2d.py) and against central finite differences of the C
oracle with the switches held fixed.

Bars: FP64 within 1e-9 of the reference (relative to its largest entry; the
nonlinear weights amplify rounding where a smoothness indicator is tiny),
FP32 within 1e-4 (the spec accuracy of the adjoint against finite
differences), directional derivatives against central differences within
1e-4 relative to their typical size."""

import numpy as np
import pytest

from gpu_util import make_pair2d, mixed_euler2d, round_to, square_domain, torch_dtype
from oracle import adjoint2d as A
from oracle import oracle as O
from paper_2002_08816_gb300 import hweno as H
from paper_2002_08816_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = [H.HWENO_FP64, H.HWENO_FP32]
TOL = {H.HWENO_FP64: 1e-9, H.HWENO_FP32: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _data(kind, nx, ny, dom, seed):
    if kind == "burgers":
        x0, x1, y0, y1 = dom
        rng = np.random.default_rng(seed)
        a = rng.uniform(0.5, 1.5)
        return W.cell_moments_2d(
            lambda x, y: 0.5 + 0.4 * np.sin(2 * np.pi * x / (x1 - x0)) * np.cos(2 * np.pi * y / (y1 - y0))
            + 0.3 * a * np.sin(4 * np.pi * (x + y) / (x1 - x0)), nx, ny, x0, x1, y0, y1, 3)
    if kind == "vortex":  # on [0, 10]^2 (nx == ny)
        return W.euler_vortex_modes_2d(nx, ny, seed=seed)
    return mixed_euler2d(nx, ny, dom, seed)


def _domain(kind, nx, ny):
    return (0.0, 10.0, 0.0, 10.0) if kind == "vortex" else square_domain(nx, ny)


def _gpu_rhs_vjp(cfg, u, flags, ax, ay, lam):
    import torch
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dt = torch_dtype(cfg.precision)
        uin = torch.from_numpy(np.ascontiguousarray(u)).to("cuda", dt)
        lin = torch.from_numpy(np.ascontiguousarray(lam)).to("cuda", dt)
        fl = torch.from_numpy(np.ascontiguousarray(flags, dtype=np.uint8)).to("cuda")
        g = torch.empty_like(uin)
        H.hweno_rhs_vjp(h, uin.data_ptr(), fl.data_ptr(), ax, ay, lin.data_ptr(), g.data_ptr())
        torch.cuda.synchronize()
        return g.double().cpu().numpy()
    finally:
        H.hweno_destroy(h)


CASES = [("burgers", H.HWENO_BURGERS), ("euler", H.HWENO_EULER)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ng", [2, 3])
@pytest.mark.parametrize("frac", [0.0, 0.3, 1.0])
@pytest.mark.parametrize("kind,system", CASES)
@pytest.mark.parametrize("size", [(16, 16), (40, 24), (7, 9)])
def test_rhs_vjp(size, kind, system, frac, ng, prec):
    """(dL/du)^T lam for given troubled cells (none, a random 30 %, all) on
    tile-spanning and ragged grids."""
    nx, ny = size
    dom = _domain(kind, nx, ny)
    seed = nx + 3 * ny + int(10 * frac)
    u = round_to(prec, _data(kind, nx, ny, dom, seed))
    cfg, ocfg = make_pair2d(system, nx, ny, dom, H.HWENO_BC_PERIODIC, prec, ng=ng)
    rng = np.random.default_rng(seed)
    flags = (rng.random((ny, nx)) < frac).astype(np.uint8)
    lam = round_to(prec, rng.standard_normal(u.shape))
    ax, ay = O.alpha2d(ocfg, u)
    ref, _ = A.rhs_vjp(ocfg, u, flags, ax, ay, lam)
    got = _gpu_rhs_vjp(cfg, u, flags, ax, ay, lam)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    # with every cell troubled in FP32, the weights' derivatives (~tau/(beta +
    # eps)^2) amplify the rounding of tiny smoothness indicators a few times more
    tol = 5e-4 if (prec == H.HWENO_FP32 and frac == 1.0) else TOL[prec]
    assert err <= tol, err


def _gpu_record_backward(cfg, u, nsteps, every, grad_out, t_final=-1.0):
    import torch
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dt = torch_dtype(cfg.precision)
        uin = torch.from_numpy(np.ascontiguousarray(u)).to("cuda", dt)
        H.hweno_set_state(h, uin.data_ptr(), cfg.precision, True)
        t = H.hweno_record(h, nsteps, every, t_final)
        uN = torch.empty_like(uin)
        H.hweno_get_state(h, uN.data_ptr(), cfg.precision, True)
        go = np.ascontiguousarray(grad_out, dtype=np.float64)
        gi = np.empty_like(go)
        H.hweno_backward(h, go.ctypes.data, gi.ctypes.data, H.HWENO_FP64, False)
        # the state is not changed by the backward pass
        uN2 = torch.empty_like(uin)
        H.hweno_get_state(h, uN2.data_ptr(), cfg.precision, True)
        assert torch.equal(uN, uN2)
        return gi, uN.double().cpu().numpy(), t
    finally:
        H.hweno_destroy(h)


def _no_band(ocfg, u, tape):
    """True when no indicator of any recorded stage input lies within 1e-6
    (relative) of the threshold, so both sides hold the same troubled cells."""
    x = u
    for sw in tape:
        flags, alphas, dt = sw
        uk = x
        for s in range(3):
            _, _, fl, ind = O.rhs2d(ocfg, uk, *alphas[s])
            if np.any(np.abs(ind - ocfg.kxrcf_threshold) <= 1e-6 * ocfg.kxrcf_threshold):
                return False
            L, Wk = A.rhs_frozen(ocfg, uk, *alphas[s], fl)
            if s == 0:
                W0 = Wk
                uk = W0 + dt * L
            elif s == 1:
                uk = 0.75 * W0 + 0.25 * Wk + (0.25 * dt) * L
        x = A.frozen_step(ocfg, x, sw)
    return True


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind,system,ng,size,nsteps,every", [
    ("vortex", H.HWENO_EULER, 3, (32, 32), 6, 4),
    ("vortex", H.HWENO_EULER, 2, (40, 40), 5, 2),
    ("mixed", H.HWENO_EULER, 3, (40, 24), 4, 3),
    ("burgers", H.HWENO_BURGERS, 3, (33, 17), 5, 5),
])
def test_backward_matches_oracle_gradient(kind, system, ng, size, nsteps, every, prec):
    """Gradient of <g, u_N> through recorded steps with checkpoint segments
    (the last one partial) against the oracle's autograd gradient along the
    oracle's own run."""
    nx, ny = size
    dom = _domain(kind, nx, ny)
    u = round_to(prec, _data(kind, nx, ny, dom, 5))
    cfg, ocfg = make_pair2d(system, nx, ny, dom, H.HWENO_BC_PERIODIC, prec, ng=ng, cfl=0.4)
    uN_o, tape = A.record(ocfg, u, nsteps, 0.4)
    assert _no_band(ocfg, u, tape)
    rng = np.random.default_rng(1)
    go = rng.standard_normal(u.shape)
    ref, _ = A.gradient(ocfg, u, tape, go)
    got, uN, _ = _gpu_record_backward(cfg, u, nsteps, every, go)
    if prec == H.HWENO_FP64:
        assert np.abs(uN - uN_o).max() <= 1e-12 * np.abs(uN_o).max()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", PRECS)
def test_backward_matches_finite_differences_64(prec):
    """The FD check of the adjoint workload at 64 x 64 (vortex plus density
    modes, 2D Euler, periodic): 16 random directions, central differences of
    the C oracle with the switches held fixed, h = 1e-6 relative."""
    n = 64
    dom = (0.0, 10.0, 0.0, 10.0)
    u = round_to(prec, W.euler_vortex_modes_2d(n, n, seed=7))
    nsteps = 4
    cfg, ocfg = make_pair2d(H.HWENO_EULER, n, n, dom, H.HWENO_BC_PERIODIC, prec, ng=3, cfl=0.4)
    _, tape = A.record(ocfg, u, nsteps, 0.4)
    rng = np.random.default_rng(3)
    go = np.zeros_like(u)
    go[0, 0] = 2.0 * rng.uniform(0.5, 1.5, size=(n, n))  # like d(sum rho^2)
    got, _, _ = _gpu_record_backward(cfg, u, nsteps, 2, go)

    def J(v):
        x = v
        for sw in tape:
            x = A.frozen_step(ocfg, x, sw)
        return float((x * go).sum())

    for _ in range(16):
        d = rng.standard_normal(u.shape)
        h = 1e-6 * np.abs(u).max() / np.abs(d).max()
        fd = (J(u + h * d) - J(u - h * d)) / (2 * h)
        ad = float((got * d).sum())
        ref = max(abs(fd), np.linalg.norm(got) * np.linalg.norm(d) / np.sqrt(got.size))
        assert abs(fd - ad) <= 1e-4 * ref, (fd, ad)


def test_autograd_function_matches_backward():
    import torch
    from paper_2002_08816_gb300 import autograd as AG
    nx = ny = 32
    dom = _domain("vortex", nx, ny)
    u = _data("vortex", nx, ny, dom, 5)
    cfg, ocfg = make_pair2d(H.HWENO_EULER, nx, ny, dom, H.HWENO_BC_PERIODIC, H.HWENO_FP64, ng=3,
                            cfl=0.4)
    run = AG.HwenoRun2D(cfg)
    try:
        u0 = torch.tensor(u, device="cuda", requires_grad=True)
        uN = run(u0, nsteps=3, checkpoint_every=2)
        loss = (uN[0, 0] ** 2).sum()
        loss.backward()
        g = u0.grad.double().cpu().numpy()
    finally:
        run.close()
    uN_o, tape = A.record(ocfg, u, 3, 0.4)
    go = np.zeros_like(u)
    go[0, 0] = 2.0 * uN_o[0, 0]
    ref, _ = A.gradient(ocfg, u, tape, go)
    assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()


def test_backward_without_record_is_an_error():
    import torch
    nx = ny = 16
    dom = square_domain(nx, ny)
    cfg, _ = make_pair2d(H.HWENO_EULER, nx, ny, dom, H.HWENO_BC_PERIODIC, H.HWENO_FP64)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        g = np.zeros((4, 3, ny, nx))
        with pytest.raises(H.HwenoError) as ei:
            H.hweno_backward(h, g.ctypes.data, g.ctypes.data, H.HWENO_FP64, False)
        assert ei.value.status == H.HWENO_ERR_STATE
    finally:
        H.hweno_destroy(h)


def test_record_rejects_outflow_boundaries():
    import torch
    nx = ny = 16
    dom = square_domain(nx, ny)
    cfg, _ = make_pair2d(H.HWENO_EULER, nx, ny, dom, H.HWENO_BC_OUTFLOW, H.HWENO_FP64)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        u = np.ascontiguousarray(W.euler_vortex_modes_2d(nx, ny, seed=1))
        H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP64, False)
        with pytest.raises(H.HwenoError) as ei:
            H.hweno_record(h, 2, 1)
        assert ei.value.status == H.HWENO_ERR_ARG
    finally:
        H.hweno_destroy(h)
