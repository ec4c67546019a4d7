"""The 1D execution choices: per-stage graph launches with 128, 256 or 512
threads per CTA give bitwise the same states (the same operations on every
cell); the persistent launch with grid barriers and the resident launch
(tiles kept in shared memory for the whole run, FP32) agree with them to
rounding (their copies of the stage body may contract a few multiply-adds
differently).  hweno_autotune keeps the state and picks one of them."""

import numpy as np
import pytest

from gpu_util import mixed_burgers, mixed_euler, round_to
from paper_2002_08816_gb300 import hweno as H
from paper_2002_08816_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CHOICES = [(t, p) for p in (0, 1) for t in (128, 256, 512)]
RESIDENT = [(256, 2), (512, 2)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _run(cfg, u, nsteps, choice, t_final=-1.0, chunks=(1,)):
    import torch
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        if choice is not None:
            H.hweno_set_execution(h, *choice)
        host = np.ascontiguousarray(u, dtype=np.float64 if cfg.precision == H.HWENO_FP64 else np.float32)
        H.hweno_set_state(h, host.ctypes.data, cfg.precision, False)
        t = None
        for k in chunks:
            t = H.hweno_step(h, nsteps * k // sum(chunks), t_final)
        out = np.empty_like(host)
        H.hweno_get_state(h, out.ctypes.data, cfg.precision, False)
        return out, t, H.hweno_stats(h)
    finally:
        H.hweno_destroy(h)


@pytest.mark.parametrize("prec", [H.HWENO_FP32, H.HWENO_FP64])
@pytest.mark.parametrize("system,bc", [(H.HWENO_EULER, H.HWENO_BC_OUTFLOW),
                                       (H.HWENO_EULER, H.HWENO_BC_REFLECTIVE),
                                       (H.HWENO_BURGERS, H.HWENO_BC_PERIODIC)])
def test_choices_agree_bitwise(system, bc, prec):
    nx = 3001
    u = mixed_euler(nx, 7) if system == H.HWENO_EULER else mixed_burgers(nx, 7)
    u = round_to(prec, u)
    cfg = H.make_config(1, system, nx, bc=bc, cfl=0.5, precision=prec)
    ref, t_ref, st_ref = _run(cfg, u, 45, (256, 0))
    for ch in CHOICES + (RESIDENT if prec == H.HWENO_FP32 else []):
        got, t, st = _run(cfg, u, 45, ch, chunks=(2, 1))
        assert st["steps"] == 45, ch
        if ch[1] == 0:
            assert np.array_equal(got, ref), ch
            assert t == t_ref and st["troubled"] == st_ref["troubled"], ch
        else:
            tol = 1e-12 if prec == H.HWENO_FP64 else 1e-6
            assert np.abs(got - ref).sum() <= tol * np.abs(ref).sum(), ch
            assert abs(t - t_ref) <= tol * t_ref, ch


def test_persistent_run_clipped_to_final_time():
    """Steps past t_final do nothing in the persistent launch too."""
    nx = 400
    u = W.burgers_sine_1d(nx)
    cfg = H.make_config(1, H.HWENO_BURGERS, nx, x0=-1.0, x1=1.0, cfl=0.6, precision=H.HWENO_FP64)
    tf = 1.5 / np.pi
    ref, t_ref, _ = _run(cfg, u, 400, (256, 0), t_final=tf)
    got, t, _ = _run(cfg, u, 400, (128, 1), t_final=tf)
    assert t == t_ref == tf
    assert np.abs(got - ref).sum() <= 1e-12 * np.abs(ref).sum()


@pytest.mark.parametrize("system,bc,nx", [(H.HWENO_EULER, H.HWENO_BC_OUTFLOW, 65536),
                                          (H.HWENO_BURGERS, H.HWENO_BC_PERIODIC, 37),
                                          (H.HWENO_EULER, H.HWENO_BC_PERIODIC, 20000),
                                          (H.HWENO_EULER, H.HWENO_BC_REFLECTIVE, 6)])
def test_resident_launch_against_the_oracle_and_per_stage(system, bc, nx):
    """The resident launch (FP32) on the benchmark's 65536-cell workload, on a
    grid of a few cells per CTA with periodic wrap across CTAs, on a periodic
    Euler grid, and on a single 6-cell tile between walls: within rounding of
    the per-stage launches, and against the oracle within the FP32 target."""
    from gpu_util import make_pair
    from oracle import oracle as O
    if nx == 65536:
        u = W.euler_two_state_1d(nx, seed=20250)
    elif nx == 6:  # a gentle wave between the walls (6 cells resolve no jump)
        u = W.cell_moments_1d(lambda x: W.euler_conserved_1d(1.0 + 0.1 * np.cos(np.pi * x),
                                                             0.0 * x, 1.0 + 0 * x), nx, 0.0, 1.0)
    elif system == H.HWENO_EULER:
        u = mixed_euler(nx, 5)
    else:
        u = mixed_burgers(nx, 5)
    u = round_to(H.HWENO_FP32, u)
    cfg, ocfg = make_pair(system, nx, 0.0, 1.0, bc, H.HWENO_FP32)
    steps = 9 if nx == 65536 else 42  # divisible by the chunks (1, 2)
    ref, t_ref, st_ref = _run(cfg, u, steps, (256, 0))
    for ch in RESIDENT:
        got, t, st = _run(cfg, u, steps, ch, chunks=(1, 2))
        assert st["steps"] == steps, ch
        assert np.abs(got - ref).sum() <= 1e-6 * np.abs(ref).sum(), ch
        assert abs(t - t_ref) <= 1e-6 * t_ref, ch
        assert st["troubled"] > 0 or st_ref["troubled"] == 0
    orc, t_o, _ = O.run1d(ocfg, u, nsteps=steps, cfl=0.5)
    rel = np.abs(got - orc).sum() / np.abs(orc).sum()
    assert rel <= 1e-4, rel
    assert abs(t - t_o) <= 1e-6 * t_o


def test_resident_run_clipped_to_final_time():
    """Steps past t_final do nothing in the resident launch either, and the
    time ends exactly at t_final."""
    nx = 400
    u = round_to(H.HWENO_FP32, W.burgers_sine_1d(nx))
    cfg = H.make_config(1, H.HWENO_BURGERS, nx, x0=-1.0, x1=1.0, cfl=0.6, precision=H.HWENO_FP32)
    tf = 1.5 / np.pi
    ref, t_ref, s_ref = _run(cfg, u, 400, (256, 0), t_final=tf)
    got, t, s = _run(cfg, u, 400, (256, 2), t_final=tf, chunks=(1, 3))
    assert t == t_ref == tf
    assert s["steps"] == s_ref["steps"]
    assert np.abs(got - ref).sum() <= 1e-5 * np.abs(ref).sum()


def test_batch_choices_agree_bitwise():
    import torch
    sizes = W.batch_sizes_1d(24, seed=3, lo=40, hi=1500)
    us = [round_to(H.HWENO_FP32, W.euler_two_state_1d(n, seed=100 + b)) for b, n in enumerate(sizes)]
    flat = np.concatenate([x.reshape(-1) for x in us]).astype(np.float32)
    cfg = H.make_config(1, H.HWENO_EULER, 16, bc=H.HWENO_BC_OUTFLOW, cfl=0.5, precision=H.HWENO_FP32)
    outs = []
    for ch in [(256, 0)] + CHOICES:
        h = H.hweno_create_batch(cfg, sizes, torch.cuda.current_stream().cuda_stream)
        try:
            H.hweno_set_execution(h, *ch)
            H.hweno_set_state(h, flat.ctypes.data, H.HWENO_FP32, False)
            H.hweno_step(h, 30)
            out = np.empty_like(flat)
            H.hweno_get_state(h, out.ctypes.data, H.HWENO_FP32, False)
            outs.append(out)
        finally:
            H.hweno_destroy(h)
    for ch, o in zip([(256, 0)] + CHOICES, outs):
        if ch[1] == 0:
            assert np.array_equal(o, outs[0]), ch
        else:
            assert np.abs(o - outs[0]).sum() <= 1e-6 * np.abs(outs[0]).sum(), ch


def test_autotune_keeps_the_state_and_picks_a_choice():
    import torch
    nx = 65536
    u = W.euler_two_state_1d(nx, seed=20250).astype(np.float32)
    cfg = H.make_config(1, H.HWENO_EULER, nx, bc=H.HWENO_BC_OUTFLOW, cfl=0.5, precision=H.HWENO_FP32)
    ref, _, _ = _run(cfg, u, 20, (256, 0))
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP32, False)
        threads, persistent = H.hweno_autotune(h, 10)
        assert threads in (128, 256, 512)
        st = H.hweno_stats(h)
        assert st["steps"] == 0 and st["t"] == 0.0
        back = np.empty_like(u)
        H.hweno_get_state(h, back.ctypes.data, H.HWENO_FP32, False)
        assert np.array_equal(back, u)
        H.hweno_step(h, 20)
        H.hweno_get_state(h, back.ctypes.data, H.HWENO_FP32, False)
        if persistent:
            assert np.abs(back - ref).sum() <= 1e-6 * np.abs(ref).sum()
        else:
            assert np.array_equal(back, ref)
    finally:
        H.hweno_destroy(h)


def test_set_execution_rejects_bad_choices():
    import torch
    cfg = H.make_config(1, H.HWENO_BURGERS, 64, precision=H.HWENO_FP64)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(H.HwenoError):
            H.hweno_set_execution(h, 200, 1)
        with pytest.raises(H.HwenoError):  # the resident launch is FP32 only
            H.hweno_set_execution(h, 256, 2)
        with pytest.raises(H.HwenoError):
            H.hweno_set_execution(h, 256, 3)
    finally:
        H.hweno_destroy(h)


def test_large_grid_epilogue_agrees_with_the_warp_level_one():
    """300,000 cells: 128-thread tiles (2459 tiles) fold the wave-speed maxima
    after a CTA reduction, 256-thread tiles (1200 tiles) warp by warp; a
    maximum and an integer count do not depend on the order, so the runs are
    bitwise equal."""
    nx = 300000
    u = round_to(H.HWENO_FP32, mixed_euler(nx, 11))
    cfg = H.make_config(1, H.HWENO_EULER, nx, bc=H.HWENO_BC_OUTFLOW, cfl=0.5,
                        precision=H.HWENO_FP32)
    a, ta, sa = _run(cfg, u, 6, (128, 0))
    b, tb, sb = _run(cfg, u, 6, (256, 0))
    assert sa["troubled"] > 0 and sa["steps"] == 6
    assert np.array_equal(a, b)
    assert ta == tb and sa["troubled"] == sb["troubled"]
