"""Pins of the oracle's reference gradient (oracle/adjoint2d.py).

The torch restatement of the 2D stage is tied to the C oracle's operator with
the troubled cells given (hwo2d_rhs_fx) on random troubled sets; its autograd
vector-Jacobian product over several frozen steps is checked against central
finite differences of the C oracle's frozen steps, which share no code with
autograd; the recorded switches reproduce the C oracle's own run.
"""

import numpy as np
import pytest
import torch

from oracle import adjoint2d as A
from oracle import oracle as O
from paper_2002_08816_gb300 import workloads as W

CASES = [
    ("burgers", O.BURGERS, lambda n: W.burgers_sine_2d(n, n), (0.0, 4.0, 0.0, 4.0)),
    ("euler-vortex", O.EULER, lambda n: W.euler_vortex_modes_2d(n, n, seed=3), (0.0, 10.0, 0.0, 10.0)),
]


def _cfg(system, n, dom, ng):
    return O.Cfg2D.make(system, n, n, *dom, O.BC_PERIODIC, n_gauss=ng)


@pytest.mark.parametrize("ng", [2, 3])
@pytest.mark.parametrize("name,system,gen,dom", CASES)
def test_torch_stage_matches_c_oracle(name, system, gen, dom, ng):
    n = 14
    u = gen(n)
    cfg = _cfg(system, n, dom, ng)
    ax, ay = O.alpha2d(cfg, u)
    st = A.Stage2D(cfg)
    rng = np.random.default_rng(11)
    for frac in (0.0, 0.3, 1.0):
        fl = (rng.random((n, n)) < frac).astype(np.uint8)
        r_c, l_c = A.rhs_frozen(cfg, u, ax, ay, fl)
        L, lim = st.rhs(torch.tensor(u), fl, ax, ay)
        # the nonlinear weights amplify the rounding differences of the two
        # evaluations (matrix products here, fits there) where beta is tiny
        scale = np.abs(r_c).max()
        assert np.abs(L.numpy() - r_c).max() <= 1e-10 * scale
        assert np.abs(lim.numpy() - l_c).max() <= 1e-12 * (np.abs(u).max() + 1.0)


def test_frozen_flags_equal_kxrcf_flags_reproduce_the_operator():
    n = 14
    u = W.euler_quadrants_2d(n, n, seed=5)
    cfg = _cfg(O.EULER, n, (0.0, 10.0, 0.0, 10.0), 3)
    rhs, ulim, fl, _ = O.rhs2d(cfg, u)
    assert 0 < fl.sum() < fl.size
    ax, ay = O.alpha2d(cfg, u)
    r2, l2 = A.rhs_frozen(cfg, u, ax, ay, fl)
    assert np.array_equal(r2, rhs) and np.array_equal(l2, ulim)


def test_frozen_flags_need_periodic_boundaries():
    n = 8
    u = W.burgers_sine_2d(n, n)
    cfg = O.Cfg2D.make(O.BURGERS, n, n, 0.0, 4.0, 0.0, 4.0, O.BC_OUTFLOW)
    with pytest.raises(FloatingPointError):
        A.rhs_frozen(cfg, u, 1.0, 1.0, np.zeros((n, n), np.uint8))
    with pytest.raises(ValueError):
        A.Stage2D(cfg)


@pytest.mark.parametrize("direction", [0, 1])
def test_euler_eigen_matches_c_oracle(direction):
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho, mu, nu, p = rng.uniform(0.3, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.3, 2)
        U = np.array([rho, rho * mu, rho * nu, p / 0.4 + 0.5 * rho * (mu * mu + nu * nu)])
        R_c, L_c = O.euler2d_eigen(1.4, U, direction)
        R_t, L_t = A.euler_eigen(1.4, torch.tensor(U), direction)
        assert np.allclose(R_t.numpy(), R_c, rtol=1e-14, atol=1e-14)
        assert np.allclose(L_t.numpy(), L_c, rtol=1e-12, atol=1e-12)
        F = A.euler_flux(1.4, torch.tensor(U), direction).numpy()
        assert np.allclose(F, O.euler2d_flux(1.4, U, direction), rtol=1e-14, atol=1e-14)


def test_record_reproduces_the_oracle_run():
    n = 12
    u = W.euler_vortex_modes_2d(n, n, seed=3)
    cfg = _cfg(O.EULER, n, (0.0, 10.0, 0.0, 10.0), 3)
    uN, tape = A.record(cfg, u, 3, 0.4)
    ref, _, _ = O.run2d(cfg, u, nsteps=3, cfl=0.4)
    assert np.abs(uN - ref).max() <= 1e-14 * np.abs(ref).max()
    assert len(tape) == 3 and all(len(sw[0]) == 3 for sw in tape)
    x = u
    for sw in tape:
        x = A.frozen_step(cfg, x, sw)
    assert np.array_equal(x, uN)


def _fd_check(cfg, u, tape, seed, rel_h, tol, ndir=3):
    rng = np.random.default_rng(seed)
    go = rng.standard_normal(u.shape)
    g, _ = A.gradient(cfg, u, tape, go)

    def J(v):
        x = v
        for sw in tape:
            x = A.frozen_step(cfg, x, sw)
        return float((x * go).sum())

    for _ in range(ndir):
        d = rng.standard_normal(u.shape)
        h = rel_h * np.abs(u).max() / np.abs(d).max()
        fd = (J(u + h * d) - J(u - h * d)) / (2 * h)
        ad = float((g * d).sum())
        # relative to the typical size of a directional derivative, so that a
        # direction nearly orthogonal to the gradient does not demand more
        ref = max(abs(ad), np.linalg.norm(g) * np.linalg.norm(d) / np.sqrt(g.size))
        assert abs(fd - ad) <= tol * ref, (fd, ad, ref)


@pytest.mark.parametrize("ng", [2, 3])
@pytest.mark.parametrize("name,system,gen,dom", CASES)
def test_gradient_matches_finite_differences_smooth(name, system, gen, dom, ng):
    """No troubled cell (the linear scheme): the frozen map is smooth; central
    differences with h = 1e-5 relative agree to ~1e-9."""
    n = 12
    u = gen(n)
    cfg = _cfg(system, n, dom, ng)
    _, tape = A.record(cfg, u, 2, 0.4)
    tape = [([np.zeros((n, n), np.uint8)] * 3, al, dt) for (_, al, dt) in tape]
    _fd_check(cfg, u, tape, seed=ng, rel_h=1e-5, tol=1e-7)


@pytest.mark.parametrize("ng", [2, 3])
@pytest.mark.parametrize("name,system,gen,dom", CASES)
def test_gradient_matches_finite_differences_troubled(name, system, gen, dom, ng):
    """A random 30 % of cells troubled in every stage (limiter and HWENO on
    every path): the nonlinear weights with eps = 1e-6 have large third
    derivatives, so h = 1e-7 relative (error ~h^2 f''' well under 1e-5)."""
    n = 12
    u = gen(n)
    cfg = _cfg(system, n, dom, ng)
    _, tape = A.record(cfg, u, 2, 0.4)
    rng = np.random.default_rng(7)
    tape = [([(rng.random((n, n)) < 0.3).astype(np.uint8) for _ in range(3)], al, dt)
            for (_, al, dt) in tape]
    _fd_check(cfg, u, tape, seed=ng + 10, rel_h=1e-7, tol=1e-5)


def test_gradient_through_recorded_shocks():
    """Quadrant data with the oracle's own troubled cells (KXRCF)."""
    n = 12
    u = W.euler_quadrants_2d(n, n, seed=5)
    cfg = _cfg(O.EULER, n, (0.0, 10.0, 0.0, 10.0), 2)
    _, tape = A.record(cfg, u, 2, 0.3)
    assert sum(int(f.sum()) for sw in tape for f in sw[0]) > 0
    _fd_check(cfg, u, tape, seed=5, rel_h=1e-7, tol=1e-5)
