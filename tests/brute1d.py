"""Brute-force evaluation of the 1D operator L of Eq. (odeH), for the oracle's pins.

Zhao & Qiu, arXiv:2002.08816, Sec. 2.1, written out from its definitions in
40-digit arithmetic (mpmath), on a tiny periodic grid, independently of the
oracle's C code:

* every candidate polynomial is solved afresh from the moment conditions of
  Step 1 and Step 2.1, in the physical coordinate s = x - x_i (not the
  oracle's reference coordinate), with exactly integrated monomials;
* smoothness indicators are Eq. (GHYZ), sum_a int_{I_i} dx^(2a-1) (p^(a))^2 dx,
  integrated exactly from the derivative's coefficients;
* the nonlinear weights follow Eq. (tao5) and the combination of Step 1 /
  Step 2.1; the interface values of Step 2.2 and the interior values of
  Step 2.3 are the quintic p0 evaluated at the points;
* the troubled-cell indicator is the reading of the KXRCF reference the
  paper defers to (Krivodonova et al.): the degree-1 polynomial of each cell,
  the jump of the traces at the inflow face, normalised by h^((k+1)/2) = h =
  dx/2, the inflow boundary measure 1 and max(|ubar_i|, 1e-12);
* Euler systems: Step 1 and Step 2.1 in the characteristic fields of the
  flux Jacobian at the cell's own average (closed-form right eigenvectors,
  left ones by a 40-digit inverse);
* Lax-Friedrichs flux, four-point Gauss-Lobatto F_i, Eq. (odeH).
"""

import mpmath as mp

mp.mp.dps = 40

GL_PTS = None  # set in _gl()


def _gl():
    r = mp.sqrt(5) / 10
    return [mp.mpf(-1) / 2, -r, r, mp.mpf(1) / 2], [mp.mpf(1) / 12, mp.mpf(5) / 12,
                                                    mp.mpf(5) / 12, mp.mpf(1) / 12]


def _int_mono(k, a, b):
    """int_a^b s^k ds, exactly."""
    return (b ** (k + 1) - a ** (k + 1)) / (k + 1)


def _fit(conds, ubar, vbar, dx):
    """Coefficients c_k of p(s) = sum c_k s^k (s = x - x_i) meeting the moment
    conditions: ('A', j) averages (1/dx) int_{I_{i+j}} p dx = ubar[j],
    ('M', j) first moments (1/dx) int_{I_{i+j}} p (x - x_{i+j})/dx dx = vbar[j]."""
    n = len(conds)
    A = mp.matrix(n, n)
    rhs = mp.matrix(n, 1)
    for r, (kind, j) in enumerate(conds):
        a, b = (j - mp.mpf(1) / 2) * dx, (j + mp.mpf(1) / 2) * dx
        for k in range(n):
            if kind == "A":
                A[r, k] = _int_mono(k, a, b) / dx
            else:  # int s^k (s - j dx) / dx ds / dx
                A[r, k] = (_int_mono(k + 1, a, b) - j * dx * _int_mono(k, a, b)) / dx ** 2
        rhs[r] = ubar[j] if kind == "A" else vbar[j]
    c = mp.lu_solve(A, rhs)
    return [c[k] for k in range(n)]


def _peval(c, s):
    return mp.fsum(ck * s ** k for k, ck in enumerate(c))


def _first_moment_on_cell(c, dx):
    a, b = -dx / 2, dx / 2
    return mp.fsum(ck * _int_mono(k + 1, a, b) for k, ck in enumerate(c)) / dx ** 2


def _beta(c, dx):
    """Eq. (GHYZ) on I_i = [-dx/2, dx/2] in s."""
    total = mp.mpf(0)
    d = list(c)
    deg = len(c) - 1
    for a in range(1, deg + 1):
        d = [d[k + 1] * (k + 1) for k in range(len(d) - 1)]
        # int (sum d_k s^k)^2 ds
        sq = mp.fsum(d[p] * d[q] * _int_mono(p + q, -dx / 2, dx / 2)
                     for p in range(len(d)) for q in range(len(d)))
        total += dx ** (2 * a - 1) * sq
    return total


def _weights(gam, b, eps):
    tau = ((abs(b[0] - b[1]) + abs(b[0] - b[2])) / 2) ** 2
    wb = [gam[n] * (1 + tau / (b[n] + eps)) for n in range(3)]
    s = mp.fsum(wb)
    return [w / s for w in wb]


def _combine(gam, om, vals):
    return om[0] * (vals[0] / gam[0] - gam[1] / gam[0] * vals[1] - gam[2] / gam[0] * vals[2]) \
        + om[1] * vals[1] + om[2] * vals[2]


def limit_scalar(ub, vb, dx, gam, eps):
    """Step 1: the modified first moment of I_i; ub = {-1, 0, 1: averages},
    vb = {-1, 1: first moments}."""
    p0 = _fit([("A", -1), ("A", 0), ("A", 1), ("M", -1), ("M", 1)], ub, vb, dx)
    p1 = _fit([("A", -1), ("A", 0)], ub, vb, dx)
    p2 = _fit([("A", 0), ("A", 1)], ub, vb, dx)
    q = [_first_moment_on_cell(p, dx) for p in (p0, p1, p2)]
    b = [_beta(p, dx) for p in (p0, p1, p2)]
    return _combine(gam, _weights(gam, b, eps), q)


def recon_scalar(ub, vb, dx, gam, eps, hweno):
    """Step 2: (u^+_{i-1/2}, u_{i-sqrt5/10}, u_{i+sqrt5/10}, u^-_{i+1/2})."""
    pts, _ = _gl()
    p0 = _fit([("A", -1), ("A", 0), ("A", 1), ("M", -1), ("M", 0), ("M", 1)], ub, vb, dx)
    out = [_peval(p0, x * dx) for x in pts]
    if hweno:
        p1 = _fit([("A", -1), ("A", 0), ("M", 0)], ub, vb, dx)
        p2 = _fit([("A", 0), ("A", 1), ("M", 0)], ub, vb, dx)
        om = _weights(gam, [_beta(p, dx) for p in (p0, p1, p2)], eps)
        for k in (0, 3):
            out[k] = _combine(gam, om, [_peval(p, pts[k] * dx) for p in (p0, p1, p2)])
    return out


def euler_flux(U, gas):
    rho, m, E = U
    mu = m / rho
    p = (gas - 1) * (E - m * mu / 2)
    return [m, m * mu + p, mu * (E + p)]


def euler_eigen(U, gas):
    rho, m, E = U
    mu = m / rho
    p = (gas - 1) * (E - m * mu / 2)
    c = mp.sqrt(gas * p / rho)
    H = (E + p) / rho
    R = mp.matrix([[1, 1, 1], [mu - c, mu, mu + c], [H - mu * c, mu * mu / 2, H + mu * c]])
    return R, R ** -1


def wave_speed(U, system, gas):
    if system == 0:
        return abs(U[0])
    rho, m, E = U
    mu = m / rho
    p = (gas - 1) * (E - m * mu / 2)
    return abs(mu) + mp.sqrt(gas * p / rho)


def kxrcf(ub, vb, i, vel, dx, N):
    """The indicator of cell i for one variable (reading of the KXRCF reference):
    the degree-1 cell polynomials P_j(x) = ubar_j + 12 vbar_j (x - x_j)/dx, the
    trace jump at the inflow face, over h = dx/2 times max(|ubar_i|, 1e-12)."""
    def P(j, s):  # s = x - x_j
        return ub[j % N] + 12 * vb[j % N] * s / dx
    if vel >= 0:  # inflow through x_{i-1/2}
        jump = P(i, -dx / 2) - P(i - 1, dx / 2)
    else:
        jump = P(i, dx / 2) - P(i + 1, -dx / 2)
    nrm = max(abs(ub[i % N]), mp.mpf("1e-12"))
    return abs(jump) / ((dx / 2) * nrm)


def rhs(u, system, dx, alpha, gam, eps=1e-6, thr=1.0, gas=1.4, mode="hybrid"):
    """L(u) of Eq. (odeH) on a periodic grid; u[c][m][i] (m = 0 average, 1
    first moment).  Returns (L, flags, indicator, limited first moments)."""
    C = 1 if system == 0 else 3
    N = len(u[0][0])
    dx, alpha, eps, thr, gas = (mp.mpf(x) for x in (dx, alpha, eps, thr, gas))
    gam = [mp.mpf(g) for g in gam]
    ub = [[mp.mpf(x) for x in u[c][0]] for c in range(C)]
    vb = [[mp.mpf(x) for x in u[c][1]] for c in range(C)]

    ind, flags = [], []
    for i in range(N):
        if system == 0:
            I = kxrcf(ub[0], vb[0], i, ub[0][i], dx, N)
        else:
            vel = ub[1][i] / ub[0][i]
            I = max(kxrcf(ub[0], vb[0], i, vel, dx, N), kxrcf(ub[2], vb[2], i, vel, dx, N))
        ind.append(I)
        flags.append(1 if mode == "all" else 0 if mode == "none" else int(I > thr))

    def nb(arr, i):
        return {-1: arr[(i - 1) % N], 0: arr[i % N], 1: arr[(i + 1) % N]}

    # Step 1 (from the unmodified moments)
    vl = [list(vb[c]) for c in range(C)]
    for i in range(N):
        if not flags[i]:
            continue
        if system == 0:
            vl[0][i] = limit_scalar(nb(ub[0], i), nb(vb[0], i), dx, gam, eps)
        else:
            R, L = euler_eigen([ub[c][i] for c in range(3)], gas)
            q = []
            for f in range(3):
                wu = {j: mp.fsum(L[f, c] * ub[c][(i + j) % N] for c in range(3)) for j in (-1, 0, 1)}
                wv = {j: mp.fsum(L[f, c] * vb[c][(i + j) % N] for c in range(3)) for j in (-1, 1)}
                q.append(limit_scalar(wu, wv, dx, gam, eps))
            for c in range(3):
                vl[c][i] = mp.fsum(R[c, f] * q[f] for f in range(3))

    # Step 2: point values of every cell
    P = [[None] * N for _ in range(C)]  # P[c][i] = 4 values at the Gauss-Lobatto points
    for i in range(N):
        hw = flags[(i - 1) % N] | flags[i] | flags[(i + 1) % N]
        for c in range(C):
            P[c][i] = recon_scalar(nb(ub[c], i), nb(vl[c], i), dx, gam, eps,
                                   hw and system == 0)
        if hw and system != 0:
            R, L = euler_eigen([ub[c][i] for c in range(3)], gas)
            ch = []
            for f in range(3):
                wu = {j: mp.fsum(L[f, c] * ub[c][(i + j) % N] for c in range(3)) for j in (-1, 0, 1)}
                wv = {j: mp.fsum(L[f, c] * vl[c][(i + j) % N] for c in range(3)) for j in (-1, 0, 1)}
                ch.append(recon_scalar(wu, wv, dx, gam, eps, True))
            for c in range(3):
                P[c][i][0] = mp.fsum(R[c, f] * ch[f][0] for f in range(3))
                P[c][i][3] = mp.fsum(R[c, f] * ch[f][3] for f in range(3))

    def flux(U):
        return [U[0] * U[0] / 2] if system == 0 else euler_flux(U, gas)

    # Lax-Friedrichs flux at x_{i+1/2}: u^- from cell i, u^+ from cell i+1
    fh = []
    for i in range(N):
        a = [P[c][i][3] for c in range(C)]
        b = [P[c][(i + 1) % N][0] for c in range(C)]
        fa, fb = flux(a), flux(b)
        fh.append([(fa[c] + fb[c]) / 2 - alpha / 2 * (b[c] - a[c]) for c in range(C)])

    _, wts = _gl()
    out = [[[None] * N, [None] * N] for _ in range(C)]
    for i in range(N):
        fq = [flux([P[c][i][k] for c in range(C)]) for k in range(4)]
        for c in range(C):
            F = mp.fsum(wts[k] * fq[k][c] for k in range(4))
            fl, fr = fh[(i - 1) % N][c], fh[i][c]
            out[c][0][i] = -(fr - fl) / dx
            out[c][1][i] = -(fl + fr) / (2 * dx) + F / dx
    return out, flags, ind, vl
