"""hweno_totals: FP64 sums of the conserved quantities on the device, against
numpy sums of the state, and their conservation under periodic boundaries
(the schemes are in flux form: Eq. (odeH), Eq. (ode2))."""

import numpy as np
import pytest

from gpu_util import mixed_burgers, mixed_euler2d, square_domain
from paper_2002_08816_gb300 import hweno as H
from paper_2002_08816_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _handle(cfg, u):
    import torch
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    host = np.ascontiguousarray(u, dtype=np.float64 if cfg.precision == H.HWENO_FP64 else np.float32)
    H.hweno_set_state(h, host.ctypes.data, cfg.precision, False)
    return h, host


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-13), (H.HWENO_FP32, 2e-6)])
def test_totals_1d_conserved(prec, tol):
    nx = 1000
    u = mixed_burgers(nx, 3)
    cfg = H.make_config(1, H.HWENO_BURGERS, nx, x0=0.0, x1=1.0, bc=H.HWENO_BC_PERIODIC, cfl=0.5,
                        precision=prec)
    h, host = _handle(cfg, u)
    try:
        t0 = H.hweno_totals(h, 1)
        assert abs(t0[0] - host[0, 0].astype(np.float64).sum() / nx) <= 1e-14 * abs(t0[0])
        H.hweno_step(h, 60)
        t1 = H.hweno_totals(h, 1)
        assert H.hweno_stats(h)["troubled"] > 0
        assert abs(t1[0] - t0[0]) <= tol * abs(t0[0])
        assert H.hweno_totals(h, 1) == t1  # repeatable to the bit
    finally:
        H.hweno_destroy(h)


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 2e-6)])
def test_totals_2d_euler_conserved(prec, tol):
    nx, ny = 48, 40
    dom = square_domain(nx, ny)
    u = mixed_euler2d(nx, ny, dom, 4)
    cfg = H.make_config(2, H.HWENO_EULER, nx, ny, x0=dom[0], x1=dom[1], y0=dom[2], y1=dom[3],
                        bc=H.HWENO_BC_PERIODIC, lin_w=(0.96, 0.01, 0.01, 0.01, 0.01), cfl=0.4,
                        precision=prec)
    h, host = _handle(cfg, u)
    try:
        t0 = np.array(H.hweno_totals(h, 4))
        cell = (dom[1] - dom[0]) / nx * (dom[3] - dom[2]) / ny
        np.testing.assert_allclose(t0, host[:, 0].astype(np.float64).sum(axis=(1, 2)) * cell, rtol=1e-13)
        H.hweno_step(h, 20)
        t1 = np.array(H.hweno_totals(h, 4))
        assert np.all(np.abs(t1 - t0) <= tol * np.abs(t0).max())
    finally:
        H.hweno_destroy(h)


def test_totals_of_a_batch_per_instance():
    import torch
    sizes = [37, 250, 613]
    states = [W.euler_two_state_1d(n, seed=9 + b) for b, n in enumerate(sizes)]
    cfg = H.make_config(1, H.HWENO_EULER, 4, bc=H.HWENO_BC_OUTFLOW, precision=H.HWENO_FP64)
    h = H.hweno_create_batch(cfg, sizes, torch.cuda.current_stream().cuda_stream)
    try:
        flat = np.ascontiguousarray(np.concatenate([s.reshape(-1) for s in states]))
        H.hweno_set_state(h, flat.ctypes.data, H.HWENO_FP64, False)
        got = np.array(H.hweno_totals(h, 3 * len(sizes))).reshape(len(sizes), 3)
        for b, (n, s) in enumerate(zip(sizes, states)):
            np.testing.assert_allclose(got[b], s[:, 0].sum(axis=1) / n, rtol=1e-13)
    finally:
        H.hweno_destroy(h)
