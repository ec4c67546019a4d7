"""Pins of the 2D oracle (Zhao & Qiu, arXiv:2002.08816, Sec. 2.2).

The oracle derives the quartic p0 (constrained least squares), the four
quadratics and the Hu-Shu smoothness indicators itself; these tests check
them against exact polynomial moments computed here with numpy, the
optimality conditions of the constrained least-squares problem, an
independent integration of Eq. (2dGHYZ), symmetry, conservation, and the
paper's Tables 3 and 4.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2002_08816_gb300 import workloads as W

CELLS = {1: (-1, -1), 2: (0, -1), 3: (1, -1), 4: (-1, 0), 5: (0, 0), 6: (1, 0),
         7: (-1, 1), 8: (0, 1), 9: (1, 1)}
MOM = [2, 4, 5, 6, 8]


def _int1(k, a, b):
    return (b ** (k + 1) - a ** (k + 1)) / (k + 1)


def _moments(C, di, dj):
    """(average, x-moment, y-moment) over cell (di, dj) of sum C[a,b] xi^a eta^b."""
    avg = xm = ym = 0.0
    for (a, b), c in np.ndenumerate(C):
        if c == 0.0:
            continue
        ix = _int1(a, di - .5, di + .5)
        iy = _int1(b, dj - .5, dj + .5)
        avg += c * ix * iy
        xm += c * (_int1(a + 1, di - .5, di + .5) - di * ix) * iy
        ym += c * ix * (_int1(b + 1, dj - .5, dj + .5) - dj * iy)
    return avg, xm, ym


def _data19(C):
    m = {k: _moments(C, *CELLS[k]) for k in CELLS}
    ub = [m[k][0] for k in range(1, 10)]
    vb = [m[k][1] for k in range(1, 10)]
    wb = [m[k][2] for k in range(1, 10)]
    d = ub + [m[k][1] for k in MOM] + [m[k][2] for k in MOM]
    return np.array(ub), np.array(vb), np.array(wb), np.array(d)


def _points(ng):
    gx = [-np.sqrt(3) / 6, np.sqrt(3) / 6] if ng == 2 else [-np.sqrt(15) / 10, 0.0,
                                                             np.sqrt(15) / 10]
    pts = [(-.5, g) for g in gx] + [(.5, g) for g in gx] + [(g, -.5) for g in gx] + \
          [(g, .5) for g in gx] + [(gk, gl) for gl in gx for gk in gx]
    return pts


def _random_poly(deg, rng):
    C = np.zeros((deg + 1, deg + 1))
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            C[a, b] = rng.normal()
    return C


@pytest.mark.parametrize("ng", [2, 3])
@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4, 5])
def test_candidates_reproduce_polynomials(ng, deg):
    """Step 5.1: p0 reproduces polynomials of degree <= 4 (exact conditions
    and a zero least-squares residual), p1..p4 those of degree <= 2."""
    rng = np.random.default_rng(100 + deg)
    C = _random_poly(deg, rng)
    ub, vb, wb, _ = _data19(C)
    val, _ = O.recon_candidates2d(ub, vb, wb, ng)
    exact = np.array([np.polynomial.polynomial.polyval2d(x, y, C) for x, y in _points(ng)])
    err0 = np.max(np.abs(val[0] - exact))
    errq = np.max(np.abs(val[1:] - exact[None, :]))
    assert (err0 < 1e-11) == (deg <= 4), err0
    assert (errq < 1e-11) == (deg <= 2), errq


def test_p0_is_the_constrained_least_squares_fit():
    """p0 matches the nine averages and the centre's first moments exactly and
    minimises the squared misfit of the first moments of cells 2, 4, 6, 8 among
    all such quartics (the gradient of the misfit is orthogonal to the
    constraints' null space)."""
    rng = np.random.default_rng(7)
    mono = O.MONO2D
    def row(kind, cell):
        r = []
        for a, b in mono:
            C = np.zeros((5, 5))
            C[a, b] = 1.0
            r.append(_moments(C, *CELLS[cell])[kind])
        return np.array(r)
    E = np.array([row(0, k) for k in range(1, 10)] + [row(1, 5), row(2, 5)])
    A = np.array([row(1, k) for k in (2, 4, 6, 8)] + [row(2, k) for k in (2, 4, 6, 8)])
    _, s, vt = np.linalg.svd(E)
    null = vt[len(s):].T
    assert null.shape[1] == 4
    for _ in range(5):
        d = rng.normal(size=19)
        c = O.p0_coeffs2d(d)
        d_eq = np.concatenate([d[:9], [d[11], d[16]]])
        d_ls = np.concatenate([d[[9, 10, 12, 13]], d[[14, 15, 17, 18]]])
        np.testing.assert_allclose(E @ c, d_eq, atol=1e-12)
        grad = A.T @ (A @ c - d_ls)
        assert np.max(np.abs(null.T @ grad)) < 1e-11


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_quadratics_match_their_stencils(n):
    stencils = {1: (1, 2, 4, 5), 2: (2, 3, 5, 6), 3: (4, 5, 7, 8), 4: (5, 6, 8, 9)}
    rng = np.random.default_rng(n)
    d = rng.normal(size=19)
    c = O.quad_coeffs2d(n, d)
    C = np.zeros((3, 3))
    for (a, b), v in zip(O.MONO2D[:6], c):
        C[a, b] = v
    for k in stencils[n]:
        assert abs(_moments(C, *CELLS[k])[0] - d[k - 1]) < 1e-12
    m5 = _moments(C, 0, 0)
    assert abs(m5[1] - d[11]) < 1e-12 and abs(m5[2] - d[16]) < 1e-12


@pytest.mark.parametrize("degree", [2, 4])
@pytest.mark.parametrize("ratio", [1.0, 2.0])
def test_hu_shu_smoothness_indicator(degree, ratio):
    """Eq. (2dGHYZ) integrated independently: numpy derivatives of the
    polynomial in physical coordinates (dx = 1, dy = ratio) and a tensor
    Gauss-Legendre rule exact for the squared derivatives."""
    rng = np.random.default_rng(degree * 10 + int(ratio))
    nm = 15 if degree == 4 else 6
    c = rng.normal(size=nm)
    P = np.zeros((5, 5))
    for (a, b), v in zip(O.MONO2D[:nm], c):
        P[a, b] = v
    dx, dy = 1.0, ratio
    # physical polynomial q(x, y) = P(x/dx, y/dy) on [-dx/2, dx/2] x [-dy/2, dy/2]
    Q = np.array([[P[a, b] / dx ** a / dy ** b for b in range(5)] for a in range(5)])
    xg, wg = np.polynomial.legendre.leggauss(8)
    X, Y = np.meshgrid(0.5 * dx * xg, 0.5 * dy * xg, indexing="ij")
    Wt = np.outer(0.5 * dx * wg, 0.5 * dy * wg)
    area = dx * dy
    want = 0.0
    for l1 in range(degree + 1):
        for l2 in range(degree + 1 - l1):
            if l1 + l2 == 0:
                continue
            D = np.polynomial.polynomial.polyder(Q, l1, axis=0) if l1 else Q
            D = np.polynomial.polynomial.polyder(D, l2, axis=1) if l2 else D
            vals = np.polynomial.polynomial.polyval2d(X, Y, D)
            want += area ** (l1 + l2 - 1) * np.sum(Wt * vals ** 2)
    got = O.beta_of_coeffs2d(degree, c, ratio)
    assert abs(got - want) <= 1e-11 * max(1.0, want)


def test_euler2d_eigenvectors():
    g = 1.4
    U = W.euler_conserved_2d(np.array(0.7), np.array(0.3), np.array(-0.5), np.array(0.9))
    rho, mu, nu = U[0], U[1] / U[0], U[2] / U[0]
    p = (g - 1) * (U[3] - 0.5 * rho * (mu * mu + nu * nu))
    c = np.sqrt(g * p / rho)
    for direction, v in ((0, mu), (1, nu)):
        R, L = O.euler2d_eigen(g, U, direction)
        h = 1e-6
        J = np.zeros((4, 4))
        for k in range(4):
            e = np.zeros(4)
            e[k] = h
            J[:, k] = (O.euler2d_flux(g, U + e, direction) - O.euler2d_flux(g, U - e, direction)) / (2 * h)
        lam = np.array([v - c, v, v, v + c])
        np.testing.assert_allclose(J @ R, R * lam[None, :], atol=1e-7)
        np.testing.assert_allclose(L @ R, np.eye(4), atol=1e-12)


def _transpose_state(u):
    """x <-> y: transpose every field, swap the x- and y-moments and (Euler)
    the two momenta."""
    t = np.transpose(u, (0, 1, 3, 2)).copy()
    t[:, [1, 2]] = t[:, [2, 1]]
    if u.shape[0] == 4:
        t[[1, 2]] = t[[2, 1]]
    return t


@pytest.mark.parametrize("system", [O.BURGERS, O.EULER])
def test_xy_symmetry(system):
    """Eq. (ode2) treats x and y alike: the right-hand side of the transposed
    state is the transposed right-hand side, troubled cells included."""
    n = 12
    if system == O.EULER:
        u = W.euler_quadrants_2d(n, n, seed=3, npts=3)
    else:
        u = W.cell_moments_2d(lambda x, y: 0.5 + np.sin(np.pi * x) * np.cos(2 * np.pi * y)
                              + (x > 0.4), n, n, 0, 1, 0, 1, 3)
    cfg = O.Cfg2D.make(system, n, n, 0, 1, 0, 1, O.BC_PERIODIC)
    r, _, fl, _ = O.rhs2d(cfg, u)
    rt, _, flt, _ = O.rhs2d(cfg, _transpose_state(u))
    assert fl.sum() > 0
    np.testing.assert_array_equal(flt, fl.T)
    np.testing.assert_allclose(rt, _transpose_state(r), rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("system", [O.BURGERS, O.EULER])
def test_constant_state_and_conservation(system):
    n = 10
    C = 4 if system == O.EULER else 1
    u = np.zeros((C, 3, n, n))
    if system == O.EULER:
        u[:, 0] = W.euler_conserved_2d(np.array(0.8), np.array(0.2), np.array(-0.3),
                                       np.array(0.6))[:, None, None]
    else:
        u[0, 0] = 0.7
    cfg = O.Cfg2D.make(system, n, n, 0, 1, 0, 1, O.BC_PERIODIC, troubled_mode=O.TROUBLED_ALL)
    r, ulim, _, _ = O.rhs2d(cfg, u)
    assert np.max(np.abs(r)) < 1e-12 and np.max(np.abs(ulim[:, 1:])) < 1e-14
    if system == O.EULER:
        u = W.euler_quadrants_2d(16, 16, seed=9, npts=3)
    else:
        u = W.cell_moments_2d(lambda x, y: 0.5 + (x > 0.5) * (y > 0.3), 16, 16, 0, 1, 0, 1, 3)
    cfg = O.Cfg2D.make(system, 16, 16, 0, 1, 0, 1, O.BC_PERIODIC)
    s0 = u[:, 0].sum(axis=(1, 2))
    u1, _, nt = O.run2d(cfg, u, nsteps=8, cfl=0.4)
    assert nt > 0
    np.testing.assert_allclose(u1[:, 0].sum(axis=(1, 2)), s0, rtol=1e-13, atol=1e-12)


def test_no_troubled_cells_on_smooth_2d_data():
    for nx in (20, 40):
        cfg = O.Cfg2D.make(O.EULER, nx, nx, 0, 2, 0, 2, O.BC_PERIODIC)
        assert O.rhs2d(cfg, W.euler_density_wave_2d(nx, nx))[2].sum() == 0
        cfg = O.Cfg2D.make(O.BURGERS, nx, nx, 0, 4, 0, 4, O.BC_PERIODIC)
        assert O.rhs2d(cfg, W.burgers_sine_2d(nx, nx))[2].sum() == 0


def _burgers2d_exact(x, y, t):
    s = x + y
    u = 0.5 + np.sin(np.pi * s / 2)
    for _ in range(100):
        g = u - (0.5 + np.sin(np.pi * (s - 2 * u * t) / 2))
        dg = 1 + np.pi * t * np.cos(np.pi * (s - 2 * u * t) / 2)
        u = u - g / dg
    return u


def test_table3_burgers2d():
    """Table 3 (Example 3.3), new hybrid HWENO at 40 x 40: L1 = 2.70E-06."""
    T = 0.5 / np.pi
    errs = {}
    for nx in (20, 40):
        dx = 4.0 / nx
        cfg = O.Cfg2D.make(O.BURGERS, nx, nx, 0, 4, 0, 4, O.BC_PERIODIC)
        u, t, nt = O.run2d(cfg, W.burgers_sine_2d(nx, nx), t_final=T,
                           dt_fixed=0.2 * dx ** (5.0 / 3.0))
        assert nt == 0 and abs(t - T) < 1e-14
        ex = W.cell_moments_2d(lambda x, y: _burgers2d_exact(x, y, T), nx, nx, 0, 4, 0, 4, 6)
        errs[nx] = np.mean(np.abs(u[0, 0] - ex[0, 0]))
    assert 2.70e-6 / 1.3 < errs[40] < 1.3 * 2.70e-6
    assert np.log(errs[20] / errs[40]) / np.log(2) > 3.5


def test_example_3_9_shocked_burgers2d():
    """Example 3.9: Example 3.3's data to T = 1.5/pi, past the shock.  The
    solution is w((x + y)/2, T) with w the entropy solution of the 1D problem
    v_t + v v_x = 0, v0 = 0.5 + sin(pi x) (Hopf-Lax, helpers.burgers_entropy_1d).
    The paper shows figures only, so the pins are convergence to the entropy
    solution: away from the shock line (more than 3 cells in x + y) the error
    falls from 2.0e-4 to 6.4e-5 (N = 20 -> 40; measured), the troubled cells
    sit on the shock line, and the overall L1 error is O(dx) from the shock."""
    from helpers import burgers_entropy_1d
    T = 1.5 / np.pi
    sv = np.linspace(0.0, 2.0, 20001)
    ws = burgers_entropy_1d(sv, T)
    s_shock = sv[np.argmin(np.diff(ws))]
    far_max = {}
    for nx in (20, 40):
        cfg = O.Cfg2D.make(O.BURGERS, nx, nx, 0, 4, 0, 4, O.BC_PERIODIC)
        u, t, nt = O.run2d(cfg, W.burgers_sine_2d(nx, nx), t_final=T, cfl=0.6)
        assert abs(t - T) < 1e-14 and nt > 0
        h, K = 4.0 / nx, 24
        off = (np.arange(K) + 0.5) / K * h
        xc = np.arange(nx) * h
        X = xc[None, :, None, None] + off[None, None, None, :]
        Y = xc[:, None, None, None] + off[None, None, :, None]
        ex = np.interp(np.mod((X + Y) / 2.0, 2.0), sv, ws).mean(axis=(2, 3))  # [j][i]
        err = np.abs(u[0, 0] - ex)
        sig = (xc[None, :] + xc[:, None] + h) / 2.0
        dist = np.abs(((sig - s_shock + 1.0) % 2.0) - 1.0)
        far = dist > 3 * h
        far_max[nx] = err[far].max()
        assert err.mean() < 1e-2
        _, _, fl, _ = O.rhs2d(cfg, u)
        assert fl.sum() > 0 and np.all(dist[fl.astype(bool)] < 4 * h)
    assert far_max[20] < 4e-4 and far_max[40] < 1.3e-4 and far_max[40] < far_max[20] / 2.5, far_max


def test_table4_euler2d():
    """Table 4 (Example 3.4), new hybrid HWENO at 30 x 30: L1 = 3.11E-07, with
    the time step small enough that the spatial error dominates."""
    T = 2.0
    errs = {}
    for nx in (20, 30):
        dx = 2.0 / nx
        cfg = O.Cfg2D.make(O.EULER, nx, nx, 0, 2, 0, 2, O.BC_PERIODIC)
        u, t, nt = O.run2d(cfg, W.euler_density_wave_2d(nx, nx), t_final=T,
                           dt_fixed=0.075 * dx ** (5.0 / 3.0))
        assert nt == 0
        ex = W.cell_moments_2d(lambda x, y: 1 + 0.2 * np.sin(np.pi * (x + y - 2 * T)),
                               nx, nx, 0, 2, 0, 2, 6)
        errs[nx] = np.mean(np.abs(u[0, 0] - ex[0, 0]))
    assert 3.11e-7 / 1.3 < errs[30] < 1.3 * 3.11e-7
    assert np.log(errs[20] / errs[30]) / np.log(1.5) > 5.5


def test_hybrid_switch_and_nonlinear_weights_2d():
    """Step 5: a cell takes HWENO values at its interface points when any cell
    of its 3x3 stencil is troubled, with tau of Eq. (tao4) and the weights of
    Eq. (99) written out here; interior points always take the linear p0."""
    n, ng = 14, 3
    u = W.cell_moments_2d(lambda x, y: 0.6 + 0.2 * np.sin(2 * np.pi * y) + (x > 0.45) * (y > 0.3),
                          n, n, 0, 1, 0, 1, 3)
    gam = np.array([0.9, 0.02, 0.03, 0.01, 0.04])
    cfg = O.Cfg2D.make(O.BURGERS, n, n, 0, 1, 0, 1, O.BC_PERIODIC, lin_w=gam)
    _, ulim, fl, _, pts = O.rhs2d(cfg, u, points=True)
    assert 0 < fl.sum() < n * n // 3
    nhw = 0
    for j in range(n):
        for i in range(n):
            cells = [((j + dj) % n, (i + di) % n) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
            hw = any(fl[c] for c in cells)
            nhw += hw
            ub = np.array([ulim[0, 0][c] for c in cells])
            vb = np.array([ulim[0, 1][c] for c in cells])
            wb = np.array([ulim[0, 2][c] for c in cells])
            val, beta = O.recon_candidates2d(ub, vb, wb, ng)
            want = val[0].copy()
            if hw:
                tau = (np.sum(np.abs(beta[0] - beta[1:])) / 4.0) ** 2
                wbar = gam * (1.0 + tau / (beta + 1e-6))
                om = wbar / wbar.sum()
                face = slice(0, 4 * ng)
                want[face] = (om[0] * (val[0, face] / gam[0]
                                       - np.sum(gam[1:, None] / gam[0] * val[1:, face], axis=0))
                              + np.sum(om[1:, None] * val[1:, face], axis=0))
            np.testing.assert_allclose(pts[0, :, j, i], want, rtol=1e-12, atol=1e-12)
    assert nhw > fl.sum()


# ----------------------------------------------------------------------------- KXRCF

def _kxrcf2d_exact(u, c, i, j, velx, vely, dx, dy):
    """The reading of the 2D KXRCF indicator in exact rationals (h by a 40-digit
    square root): the degree-1 cell polynomial P(x, y) = ubar + 12 vbar (x -
    x_i)/dx + 12 wbar (y - y_j)/dy, the trace differences P_cell - P_nb
    integrated exactly along the inflow x-face (left when velx >= 0) and the
    inflow y-face (bottom when vely >= 0), the absolute value of their sum over
    h |dI^-| max(|ubar|, 1e-12), h = sqrt(dx^2 + dy^2)/2 (half the diagonal),
    |dI^-| = dy + dx (the inflow boundary's length)."""
    from fractions import Fraction as Fr
    import mpmath as mp
    ny, nx = u.shape[2], u.shape[3]
    dxf, dyf = Fr(dx), Fr(dy)

    def coef(ci, cj):
        ci, cj = ci % nx, cj % ny
        return Fr(u[c, 0, cj, ci]), Fr(u[c, 1, cj, ci]), Fr(u[c, 2, cj, ci])

    def P(ci, cj, sx, sy):  # sx = x - x_ci, sy = y - y_cj
        a, v, w = coef(ci, cj)
        return a + 12 * v * sx / dxf + 12 * w * sy / dyf

    def line_int(f, t0, t1):
        # f linear in t: the trapezoid rule is exact
        return (f(t0) + f(t1)) / 2 * (t1 - t0)

    hx, hy = dxf / 2, dyf / 2
    if velx >= 0:   # face x = x_{i-1/2}: the cell at sx = -hx, the left neighbour at +hx
        ix = line_int(lambda t: P(i, j, -hx, t) - P(i - 1, j, hx, t), -hy, hy)
    else:
        ix = line_int(lambda t: P(i, j, hx, t) - P(i + 1, j, -hx, t), -hy, hy)
    if vely >= 0:
        iy = line_int(lambda t: P(i, j, t, -hy) - P(i, j - 1, t, hy), -hx, hx)
    else:
        iy = line_int(lambda t: P(i, j, t, hy) - P(i, j + 1, t, -hy), -hx, hx)
    nrm = max(abs(Fr(u[c, 0, j % ny, i % nx])), Fr(1e-12))
    q = abs(ix + iy) / ((dxf + dyf) * nrm)
    mp.mp.dps = 40
    h = mp.sqrt(mp.mpf(dx) ** 2 + mp.mpf(dy) ** 2) / 2
    return float(mp.mpf(q.numerator) / mp.mpf(q.denominator) / h)


def test_kxrcf_indicator_hand_computed_2d():
    """Sec. 2.2 Step 4 / Remark 3 (KXRCF, reading of the deferred reference):
    the oracle's indicator equals the exact value on small periodic grids with
    dx != dy, for Burgers (velocity (u, u): both signs occur) and for Euler
    through rho and E with the velocity (m/rho, n/rho) of the cell (all four
    sign pairs occur), so both face pairs and both sides of each are used."""
    rng = np.random.default_rng(5)
    nx, ny, dx, dy = 4, 3, 0.25, 0.4
    u = np.zeros((1, 3, ny, nx))
    u[0, 0] = rng.uniform(-1, 1, (ny, nx))
    u[0, 1:] = rng.uniform(-0.1, 0.1, (2, ny, nx))
    cfg = O.Cfg2D.make(O.BURGERS, nx, ny, 0.0, nx * dx, 0.0, ny * dy, O.BC_PERIODIC)
    _, _, flags, ind = O.rhs2d(cfg, u, 2.0, 2.0)
    signs = set()
    for j in range(ny):
        for i in range(nx):
            v = u[0, 0, j, i]
            want = _kxrcf2d_exact(u, 0, i, j, v, v, dx, dy)
            assert abs(ind[j, i] - want) <= 1e-13 * want, (i, j, ind[j, i], want)
            assert flags[j, i] == (want > 1.0)
            signs.add(v >= 0)
    assert signs == {True, False}
    # Euler
    rho = rng.uniform(0.5, 1.5, (ny, nx))
    mu = rng.choice([-1, 1], (ny, nx)) * rng.uniform(0.1, 0.5, (ny, nx))
    nu = rng.choice([-1, 1], (ny, nx)) * rng.uniform(0.1, 0.5, (ny, nx))
    mu[0, :2], nu[0, :2] = [0.3, -0.3], [0.2, 0.2]
    mu[1, :2], nu[1, :2] = [0.3, -0.3], [-0.2, -0.2]
    p = rng.uniform(0.5, 1.5, (ny, nx))
    u = np.zeros((4, 3, ny, nx))
    u[:, 0] = W.euler_conserved_2d(rho, mu, nu, p)
    u[:, 1:] = rng.uniform(-0.03, 0.03, (4, 2, ny, nx))
    cfg = O.Cfg2D.make(O.EULER, nx, ny, 0.0, nx * dx, 0.0, ny * dy, O.BC_PERIODIC)
    _, _, flags, ind = O.rhs2d(cfg, u, 3.0, 3.0)
    pairs = set()
    for j in range(ny):
        for i in range(nx):
            vx = u[1, 0, j, i] / u[0, 0, j, i]
            vy = u[2, 0, j, i] / u[0, 0, j, i]
            want = max(_kxrcf2d_exact(u, 0, i, j, vx, vy, dx, dy),
                       _kxrcf2d_exact(u, 3, i, j, vx, vy, dx, dy))
            assert abs(ind[j, i] - want) <= 1e-13 * want, (i, j)
            assert flags[j, i] == (want > 1.0)
            pairs.add((vx >= 0, vy >= 0))
    assert len(pairs) == 4


def test_kxrcf_scaling_laws_2d():
    """The 2D normalisation h |dI^-| (h the half diagonal): on smooth data the
    face-integrated jump is O(dx^4) (O(dx^3) per unit length by the same
    projection symmetry as in 1D, times the face length), the denominator
    O(dx^2), so the indicator falls like dx^2; across a discontinuity aligned
    with the x-faces it grows like 1/dx, with the value fixed by the
    normalisation: I = |jump| dy / (sqrt(2) dx/2 * 2 dx * |u|) on square cells."""
    def ind_of(func, n):
        u = W.cell_moments_2d(func, n, n, 0.0, 1.0, 0.0, 1.0, 3)
        cfg = O.Cfg2D.make(O.BURGERS, n, n, 0.0, 1.0, 0.0, 1.0, O.BC_PERIODIC)
        _, _, _, ind = O.rhs2d(cfg, u, 3.0, 3.0)
        return ind
    smooth = lambda x, y: 1.5 + 0.3 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    a, b = ind_of(smooth, 16).max(), ind_of(smooth, 32).max()
    order = np.log2(a / b)
    assert 1.7 < order < 2.3, order
    step = lambda x, y: np.where((x > 0.25) & (x < 0.75), 1.0, 0.5) + 0 * y
    for n in (16, 32):
        ind = ind_of(step, n)
        dx = 1.0 / n
        want = 0.5 * dx / (np.sqrt(2) * dx / 2 * 2 * dx * 1.0)  # rising face, u = 1
        np.testing.assert_allclose(ind[:, n // 4], want, rtol=1e-12)
        np.testing.assert_allclose(ind[:, 3 * n // 4], 2 * want, rtol=1e-12)
