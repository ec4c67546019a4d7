"""Failure detection on the GPU without a fault: the bounded grid barrier of
the persistent launch gives up when an arrival never comes (a counter that
nothing completes), records the timeout in a status word the host reads, and
leaves the context usable."""

import time

import numpy as np
import pytest

from gpu_util import mixed_euler
from paper_2002_08816_gb300 import hweno as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def test_barrier_meetings_complete_when_every_cta_arrives():
    assert H.hweno_check_barrier(8, 200, 0, 1 << 20) == H.HWENO_OK
    assert H.hweno_check_barrier(152, 50, 0, 1 << 20) == H.HWENO_OK


def test_lost_arrival_times_out_and_the_context_stays_usable():
    t0 = time.time()
    assert H.hweno_check_barrier(8, 3, 1, 2000) == H.HWENO_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    # the same process keeps working: a persistent run and a graph run agree
    import torch
    nx = 1000
    u = mixed_euler(nx, 3).astype(np.float32)
    cfg = H.make_config(1, H.HWENO_EULER, nx, bc=H.HWENO_BC_OUTFLOW, cfl=0.5,
                        precision=H.HWENO_FP32)
    out = []
    for persistent in (0, 1):
        h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
        try:
            H.hweno_set_execution(h, 256, persistent)
            H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP32, False)
            H.hweno_step(h, 10)
            o = np.empty_like(u)
            H.hweno_get_state(h, o.ctypes.data, H.HWENO_FP32, False)
            out.append(o)
        finally:
            H.hweno_destroy(h)
    assert np.all(np.isfinite(out[1]))
    assert np.abs(out[0] - out[1]).sum() <= 1e-6 * np.abs(out[0]).sum()
    assert H.hweno_check_barrier(8, 10, 0, 1 << 20) == H.HWENO_OK


def test_resident_launch_gives_up_when_a_cta_never_publishes():
    """The resident launch's waits are bounded: with one CTA that never
    publishes its maximum no CTA can form alpha, every wait runs out (2^14
    polls here), the host reads HWENO_ERR_TIMEOUT, the state is left as it was,
    and the handle then runs ordinary resident steps that agree with the
    per-stage launches."""
    import torch
    nx = 65536
    u = mixed_euler(nx, 4).astype(np.float32)
    cfg = H.make_config(1, H.HWENO_EULER, nx, bc=H.HWENO_BC_OUTFLOW, cfl=0.5,
                        precision=H.HWENO_FP32)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        H.hweno_set_execution(h, 256, 2)
        H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP32, False)
        assert H.hweno_check_resident(h, 3, -1, 1 << 21) == H.HWENO_OK  # no silent CTA
        H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP32, False)
        t0 = time.time()
        assert H.hweno_check_resident(h, 3, 17, 1 << 14) == H.HWENO_ERR_TIMEOUT
        assert time.time() - t0 < 30.0
        back = np.empty_like(u)
        H.hweno_get_state(h, back.ctypes.data, H.HWENO_FP32, False)
        assert np.array_equal(back, u)  # an aborted run writes nothing
        H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP32, False)  # resets the status
        H.hweno_step(h, 10)
        got = np.empty_like(u)
        H.hweno_get_state(h, got.ctypes.data, H.HWENO_FP32, False)
    finally:
        H.hweno_destroy(h)
    h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        H.hweno_set_state(h, u.ctypes.data, H.HWENO_FP32, False)
        H.hweno_step(h, 10)
        ref = np.empty_like(u)
        H.hweno_get_state(h, ref.ctypes.data, H.HWENO_FP32, False)
    finally:
        H.hweno_destroy(h)
    assert np.abs(got - ref).sum() <= 1e-6 * np.abs(ref).sum()
