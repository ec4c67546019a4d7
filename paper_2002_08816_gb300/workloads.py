"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds no arithmetic of the scheme itself: it samples initial data
(point functions of x, or x and y) and turns them into the paper's zeroth and
first moments by tensor Gauss-Legendre quadrature (the initial conditions of
Eq. (odeH) and Eq. (ode2)).  Both the CUDA path and the oracle consume its
output.  Random draws use numpy's PCG64 generator with an explicit seed.

Layouts match the library: 1D ``[C][2][nx]`` and 2D ``[C][3][ny][nx]``.
"""

import numpy as np

GAMMA = 1.4


def _gauss(npts):
    xg, wg = np.polynomial.legendre.leggauss(npts)
    return 0.5 * xg, 0.5 * wg  # nodes on [-1/2, 1/2], weights summing to 1


def cell_moments_1d(func, nx, x0, x1, npts=5):
    """func(x) -> array [C, ...]; returns moments [C, 2, nx] (average, first)."""
    dx = (x1 - x0) / nx
    xc = x0 + (np.arange(nx) + 0.5) * dx
    xi, w = _gauss(npts)
    pts = xc[None, :] + xi[:, None] * dx          # [npts, nx]
    vals = np.asarray(func(pts), dtype=np.float64)  # [C, npts, nx]
    if vals.ndim == 2:
        vals = vals[None]
    avg = np.einsum("q,cqn->cn", w, vals)
    mom = np.einsum("q,cqn->cn", w * xi, vals)
    return np.stack([avg, mom], axis=1)


def cell_moments_2d(func, nx, ny, x0, x1, y0, y1, npts=5):
    """func(x, y) -> array [C, ...]; returns moments [C, 3, ny, nx]."""
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * dx
    yc = y0 + (np.arange(ny) + 0.5) * dy
    xi, w = _gauss(npts)
    C = None
    out = None
    for a in range(npts):
        for b in range(npts):
            X = xc[None, :] + xi[a] * dx
            Y = yc[:, None] + xi[b] * dy
            v = np.asarray(func(np.broadcast_to(X, (ny, nx)), np.broadcast_to(Y, (ny, nx))),
                           dtype=np.float64)
            if v.ndim == 2:
                v = v[None]
            if out is None:
                C = v.shape[0]
                out = np.zeros((C, 3, ny, nx))
            ww = w[a] * w[b]
            out[:, 0] += ww * v
            out[:, 1] += ww * xi[a] * v
            out[:, 2] += ww * xi[b] * v
    return out


# ----------------------------------------------------------------------------- physics of the data

def euler_conserved_1d(rho, mu, p, gamma=GAMMA):
    return np.stack([rho, rho * mu, p / (gamma - 1.0) + 0.5 * rho * mu * mu])


def euler_conserved_2d(rho, mu, nu, p, gamma=GAMMA):
    return np.stack([rho, rho * mu, rho * nu,
                     p / (gamma - 1.0) + 0.5 * rho * (mu * mu + nu * nu)])


# ----------------------------------------------------------------------------- 1D workloads

def burgers_sine_1d(nx, x0=-1.0, x1=1.0, npts=5):
    """Burgers u0 = 0.5 + sin(pi x), periodic (Sec. 3, Examples 3.1 and 3.5)."""
    return cell_moments_1d(lambda x: 0.5 + np.sin(np.pi * x), nx, x0, x1, npts)


def euler_density_wave_1d(nx, x0=0.0, x1=2.0, npts=5, gamma=GAMMA):
    """rho = 1 + 0.2 sin(pi x), mu = p = 1, periodic (Example 3.2)."""
    def f(x):
        return euler_conserved_1d(1.0 + 0.2 * np.sin(np.pi * x), np.ones_like(x),
                                  np.ones_like(x), gamma)
    return cell_moments_1d(f, nx, x0, x1, npts)


def euler_riemann_1d(nx, left, right, x0, x1, xs, npts=5, gamma=GAMMA):
    """Piecewise-constant (rho, mu, p) with a jump at xs."""
    def f(x):
        L = x < xs
        rho = np.where(L, left[0], right[0])
        mu = np.where(L, left[1], right[1])
        p = np.where(L, left[2], right[2])
        return euler_conserved_1d(rho, mu, p, gamma)
    return cell_moments_1d(f, nx, x0, x1, npts)


def euler_two_state_1d(nx, seed, x0=0.0, x1=1.0, npts=5, gamma=GAMMA, nmodes=4,
                       amp=0.2):
    """Seeded piecewise-smooth 1D Euler data on [0, 1] with outflow ends.

    (rho, mu, p) left and right of x = 0.5 drawn from U(0.1,1) x U(-1,1) x
    U(0.1,1); the right density carries ``nmodes`` sinusoidal modes with
    integer wave numbers in [4, 256] and random phases, averaged so that the
    total relative amplitude stays below ``amp``.
    """
    rng = np.random.default_rng(seed)
    sl = (rng.uniform(0.1, 1.0), rng.uniform(-1.0, 1.0), rng.uniform(0.1, 1.0))
    sr = (rng.uniform(0.1, 1.0), rng.uniform(-1.0, 1.0), rng.uniform(0.1, 1.0))
    k = rng.integers(4, 257, size=nmodes)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=nmodes)

    def f(x):
        L = x < 0.5
        modes = sum(np.sin(2.0 * np.pi * k[m] * x + ph[m]) for m in range(nmodes)) / nmodes
        rho = np.where(L, sl[0], sr[0] * (1.0 + amp * modes))
        mu = np.where(L, sl[1], sr[1])
        p = np.where(L, sl[2], sr[2])
        return euler_conserved_1d(rho, mu, p, gamma)

    return cell_moments_1d(f, nx, x0, x1, npts)


def euler_lax_tiled_1d(nx, cells_per_tile=800, npts=5, gamma=GAMMA):
    """The Lax problem's two states (Example 3.6: (rho, mu, p) = (0.445, 0.698,
    3.528) left of the jump, (0.5, 0, 0.571) right of it) repeated: the domain
    [0, 1] holds nx / cells_per_tile copies of one Lax problem, each on
    cells_per_tile cells with its jump in the middle, so that the share of
    troubled cells resembles the paper's shock tests (3.5-14 %) rather than
    one shock on a fine grid: 800 cells per copy give about 10 % over 200
    steps with periodic ends."""
    ntile = max(1, nx // cells_per_tile)

    def f(x):
        frac = (x * ntile) % 1.0
        L = frac < 0.5
        rho = np.where(L, 0.445, 0.5)
        mu = np.where(L, 0.698, 0.0)
        p = np.where(L, 3.528, 0.571)
        return euler_conserved_1d(rho, mu, p, gamma)

    return cell_moments_1d(f, nx, 0.0, 1.0, npts)


def batch_sizes_1d(n_instances, seed, lo=256, hi=16384):
    """Cell counts log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_instances))).astype(np.int64)


def random_lin_weights(nsteps, ncand, seed, lo=0.01, hi=1.0):
    """gamma_n = r_n / sum r, r_n ~ U(lo, hi), one set per time step."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(lo, hi, size=(nsteps, ncand))
    return r / r.sum(axis=1, keepdims=True)


# ----------------------------------------------------------------------------- 2D workloads

def burgers_sine_2d(nx, ny, npts=5):
    """u0 = 0.5 + sin(pi (x + y)/2) on [0, 4]^2, periodic (Example 3.3)."""
    return cell_moments_2d(lambda x, y: 0.5 + np.sin(np.pi * (x + y) / 2.0),
                           nx, ny, 0.0, 4.0, 0.0, 4.0, npts)


def euler_density_wave_2d(nx, ny, npts=5, gamma=GAMMA):
    """rho = 1 + 0.2 sin(pi (x + y)), mu = nu = p = 1 on [0, 2]^2 (Example 3.4)."""
    def f(x, y):
        one = np.ones_like(x)
        return euler_conserved_2d(1.0 + 0.2 * np.sin(np.pi * (x + y)), one, one, one, gamma)
    return cell_moments_2d(f, nx, ny, 0.0, 2.0, 0.0, 2.0, npts)


def euler_vortex_modes_2d(nx, ny, seed, L=10.0, strength=5.0, nmodes=8, amp=0.05,
                          npts=3, gamma=GAMMA):
    """Uniform flow (1,1,1,1) + isentropic vortex + seeded density modes, periodic [0,L]^2."""
    rng = np.random.default_rng(seed)
    a = rng.integers(1, 17, size=nmodes)
    b = rng.integers(1, 17, size=nmodes)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=nmodes)

    def f(x, y):
        xb, yb = x - 0.5 * L, y - 0.5 * L
        r2 = xb * xb + yb * yb
        e = strength / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
        mu = 1.0 - e * yb
        nu = 1.0 + e * xb
        T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
        rho = T ** (1.0 / (gamma - 1.0))
        p = rho ** gamma
        modes = sum(np.sin(2.0 * np.pi * (a[m] * x + b[m] * y) / L + ph[m])
                    for m in range(nmodes)) / nmodes
        rho = rho * (1.0 + amp * modes)
        return euler_conserved_2d(rho, mu, nu, p, gamma)

    return cell_moments_2d(f, nx, ny, 0.0, L, 0.0, L, npts)


def euler_quadrants_2d(nx, ny, seed, L=10.0, npts=3, gamma=GAMMA):
    """Four constant quadrants split at (L/2, L/2), states drawn from the seed."""
    rng = np.random.default_rng(seed)
    st = [(rng.uniform(0.1, 1.0), rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0),
           rng.uniform(0.1, 1.0)) for _ in range(4)]

    def f(x, y):
        q = (x >= 0.5 * L).astype(int) + 2 * (y >= 0.5 * L).astype(int)
        comp = [np.choose(q, [s[k] for s in st]) for k in range(4)]
        return euler_conserved_2d(comp[0], comp[1], comp[2], comp[3], gamma)

    return cell_moments_2d(f, nx, ny, 0.0, L, 0.0, L, npts)
