"""hweno_rhs1d_noalloc, the allocation-free 1D right-hand side, against
hweno_rhs.

The entry point exists for callers that cannot let the library call
cudaMalloc (device memory owned by the caller's own pool allocator, budgeted
allocations, or loops that cannot afford the synchronisation an allocation
may cause); it keeps its scratch in a fixed __device__ array instead.  This
file runs last (pytest collects it after the other test files) and passes
both alone in a fresh process and after the whole suite.
"""

import numpy as np
import pytest

from gpu_util import (band_cells, make_pair, mixed_burgers, mixed_euler, rhs_tolerance,
                      round_to)
from oracle import oracle as O
from paper_2002_08816_gb300 import hweno as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()


def _both(system, nx, bc, prec, u):
    """L(u) from hweno_rhs (handle with its own cudaMalloc'd scratch) and from
    hweno_rhs1d_noalloc (fixed scratch), on the same device input."""
    import torch
    cfg, ocfg = make_pair(system, nx, 0.0, 1.0, bc, prec)
    stream = torch.cuda.current_stream().cuda_stream
    dt = torch.float64 if prec == H.HWENO_FP64 else torch.float32
    uin = torch.from_numpy(np.ascontiguousarray(u)).to("cuda", dt)
    ref_out, ref_lim = torch.empty_like(uin), torch.empty_like(uin)
    ref_fl = torch.zeros(nx, dtype=torch.uint8, device="cuda")
    h = H.hweno_create(cfg, stream)
    try:
        H.hweno_rhs(h, uin.data_ptr(), ref_out.data_ptr(), ref_fl.data_ptr(), ref_lim.data_ptr())
    finally:
        H.hweno_destroy(h)
    out, lim = torch.full_like(uin, float("nan")), torch.full_like(uin, float("nan"))
    fl = torch.full((nx,), 7, dtype=torch.uint8, device="cuda")
    st = H.hweno_rhs1d_noalloc(cfg, stream, uin.data_ptr(), out.data_ptr(), fl.data_ptr(),
                               lim.data_ptr())
    torch.cuda.synchronize()
    assert st == H.HWENO_OK, st
    tol = rhs_tolerance(prec, ocfg, u)
    a, b = out.double().cpu().numpy(), ref_out.double().cpu().numpy()
    assert np.all(np.isfinite(a))
    assert np.max(np.abs(a - b)) <= tol
    assert np.max(np.abs(lim.double().cpu().numpy() - ref_lim.double().cpu().numpy())) <= tol
    assert np.array_equal(fl.cpu().numpy(), ref_fl.cpu().numpy())
    return fl.cpu().numpy(), a


@pytest.mark.parametrize("prec", [H.HWENO_FP64, H.HWENO_FP32])
def test_noalloc_matches_hweno_rhs_on_two_calls_in_a_row(prec):
    nx1, nx2 = 3001, 700
    u1 = round_to(prec, mixed_euler(nx1, 31))
    u2 = round_to(prec, mixed_burgers(nx2, 32))
    f1, _ = _both(H.HWENO_EULER, nx1, H.HWENO_BC_OUTFLOW, prec, u1)
    f2, _ = _both(H.HWENO_BURGERS, nx2, H.HWENO_BC_PERIODIC, prec, u2)
    assert f1.sum() > 0 and f2.sum() > 0  # both calls went through troubled cells


def test_noalloc_status_word_starts_clean_each_call():
    """A non-physical input sets the shared status word; the next valid call
    must not inherit it."""
    import torch
    nx = 512
    bad = mixed_euler(nx, 5)
    bad[0, 0, 100] = -1.0
    cfg, _ = make_pair(H.HWENO_EULER, nx, 0.0, 1.0, H.HWENO_BC_OUTFLOW, H.HWENO_FP64)
    stream = torch.cuda.current_stream().cuda_stream
    ub = torch.from_numpy(bad).to("cuda")
    out = torch.empty_like(ub)
    assert H.hweno_rhs1d_noalloc(cfg, stream, ub.data_ptr(), out.data_ptr()) == \
        H.HWENO_ERR_NONPHYSICAL
    _both(H.HWENO_EULER, nx, H.HWENO_BC_OUTFLOW, H.HWENO_FP64, mixed_euler(nx, 5))


def test_noalloc_rejects_more_cells_than_its_scratch_holds():
    import torch
    nx = H.HWENO_NOALLOC_MAX_CELLS + 1
    cfg, _ = make_pair(H.HWENO_BURGERS, nx, 0.0, 1.0, H.HWENO_BC_PERIODIC, H.HWENO_FP32)
    uin = torch.ones((1, 2, nx), dtype=torch.float32, device="cuda")
    out = torch.empty_like(uin)
    st = H.hweno_rhs1d_noalloc(cfg, torch.cuda.current_stream().cuda_stream, uin.data_ptr(),
                               out.data_ptr())
    assert st == H.HWENO_ERR_TOO_LARGE


@pytest.mark.parametrize("prec", [H.HWENO_FP64, H.HWENO_FP32])
def test_noalloc_reflective_walls_match_hweno_rhs_and_the_oracle(prec):
    """Reflective walls (1D Euler), a configuration hweno_create accepts, give
    the same L as hweno_rhs and as the oracle (flags bit-exact outside the
    1e-6 band around the KXRCF threshold)."""
    nx = 1000
    u = round_to(prec, mixed_euler(nx, 41))
    fl, got = _both(H.HWENO_EULER, nx, H.HWENO_BC_REFLECTIVE, prec, u)
    _, ocfg = make_pair(H.HWENO_EULER, nx, 0.0, 1.0, H.HWENO_BC_REFLECTIVE, prec)
    rhs, _, oflags, ind = O.rhs1d(ocfg, u)
    near, mask = band_cells(ind, ocfg.kxrcf_threshold, nx, periodic=False)
    assert fl.sum() > 0
    assert np.array_equal(fl[~near], oflags[~near])
    tol = rhs_tolerance(prec, ocfg, u)
    keep = ~mask
    assert np.max(np.abs(got[:, :, keep] - rhs[:, :, keep])) <= tol


def test_noalloc_rejects_what_hweno_create_rejects():
    """Unknown variant bits and a non-positive CFL number fail as in
    hweno_create; a 2D configuration is refused."""
    import torch
    nx = 64
    uin = torch.ones((1, 2, nx), dtype=torch.float64, device="cuda")
    out = torch.empty_like(uin)
    stream = torch.cuda.current_stream().cuda_stream
    for bad in ("variant", "cfl", "dim"):
        cfg, _ = make_pair(H.HWENO_BURGERS, nx, 0.0, 1.0, H.HWENO_BC_PERIODIC, H.HWENO_FP64)
        if bad == "variant":
            cfg.variant = 1 << 7
        elif bad == "cfl":
            cfg.cfl = 0.0
        else:
            cfg.dim = 2
        assert H.hweno_rhs1d_noalloc(cfg, stream, uin.data_ptr(), out.data_ptr()) == \
            H.HWENO_ERR_ARG, bad
