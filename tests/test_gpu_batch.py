"""A batch of independent 1D instances of uneven size advanced in shared
launches (hweno_create_batch) against the oracle run on each instance alone."""

import numpy as np
import pytest

from gpu_util import round_to, torch_dtype
from oracle import oracle as O
from paper_2002_08816_gb300 import hweno as H
from paper_2002_08816_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _batch_state(sizes, seed):
    return [W.euler_two_state_1d(int(n), seed=seed + b) for b, n in enumerate(sizes)]


def _run_batch(sizes, states, prec, nsteps, t_final=-1.0, cfl=0.5):
    import torch
    cfg = H.make_config(1, H.HWENO_EULER, 4, x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW, cfl=cfl,
                        precision=prec)
    h = H.hweno_create_batch(cfg, sizes, torch.cuda.current_stream().cuda_stream)
    try:
        flat = np.concatenate([s.reshape(-1) for s in states])
        dev = torch.from_numpy(flat).to("cuda", torch_dtype(prec))
        H.hweno_set_state(h, dev.data_ptr(), prec, True)
        H.hweno_step(h, nsteps, t_final)
        out = torch.empty_like(dev)
        H.hweno_get_state(h, out.data_ptr(), prec, True)
        times = H.hweno_batch_times(h, len(sizes))
        got = out.double().cpu().numpy()
    finally:
        H.hweno_destroy(h)
    res, off = [], 0
    for s in states:
        res.append(got[off:off + s.size].reshape(s.shape))
        off += s.size
    return res, times


def _oracle(n, u, nsteps, t_final=-1.0, cfl=0.5):
    ocfg = O.Cfg1D.make(O.EULER, int(n), 0.0, 1.0, O.BC_OUTFLOW)
    return O.run1d(ocfg, u, nsteps=nsteps, cfl=cfl, t_final=t_final)


@pytest.mark.parametrize("prec,tol", [(H.HWENO_FP64, 1e-12), (H.HWENO_FP32, 1e-4)])
def test_uneven_batch_matches_each_instance(prec, tol):
    sizes = [4, 5, 37, 250, 251, 777, 1000, 33, 300]
    states = [round_to(prec, s) for s in _batch_state(sizes, 40)]
    got, times = _run_batch(sizes, states, prec, 20)
    for b, n in enumerate(sizes):
        ref, t_ref, _ = _oracle(n, states[b], 20)
        rel = np.abs(got[b] - ref).sum() / np.abs(ref).sum()
        assert rel <= tol, (b, n, rel)
        # FP32: dt follows alpha = max |u| + c of an FP32 state that may differ
        # from the FP64 one by ~1e-5 relative near a shock (the state bar is
        # 1e-4 in L1), so the time after 20 steps is held to 1e-5
        assert abs(times[b] - t_ref) <= (1e-13 if prec == H.HWENO_FP64 else 1e-5) * t_ref


def test_batch_final_time_per_instance():
    """Each instance has its own dt (its own dx and alpha) and is clipped to the
    final time separately; finished instances stop while others go on."""
    sizes = [64, 300, 1200]
    states = _batch_state(sizes, 7)
    T = 0.01
    got, times = _run_batch(sizes, states, H.HWENO_FP64, 400, t_final=T)
    for b, n in enumerate(sizes):
        ref, t_ref, _ = _oracle(n, states[b], 400, t_final=T)
        assert times[b] == T and t_ref == T
        assert np.abs(got[b] - ref).sum() / np.abs(ref).sum() <= 1e-12


def test_512_instance_workload_fp32_sampled():
    """The batched workload: 512 instances with cell counts log-uniform in
    [256, 16384], two-state data, FP32; 6 steps, 10 instances checked."""
    sizes = W.batch_sizes_1d(512, seed=77)
    states = [s.astype(np.float32).astype(np.float64) for s in _batch_state(sizes, 1000)]
    got, times = _run_batch([int(v) for v in sizes], states, H.HWENO_FP32, 6)
    rng = np.random.default_rng(3)
    for b in list(rng.choice(512, size=8, replace=False)) + [int(np.argmax(sizes)), int(np.argmin(sizes))]:
        ref, t_ref, _ = _oracle(sizes[b], states[b], 6)
        rel = np.abs(got[b] - ref).sum() / np.abs(ref).sum()
        assert rel <= 1e-4, (b, sizes[b], rel)
        assert abs(times[b] - t_ref) <= 1e-6 * t_ref
