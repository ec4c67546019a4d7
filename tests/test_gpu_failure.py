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
