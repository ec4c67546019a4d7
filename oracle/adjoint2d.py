"""ORACLE -- test infrastructure only.

Reference gradient of the 2D hybrid HWENO scheme (Zhao & Qiu,
arXiv:2002.08816, Sec. 2.2) with its switches held fixed.

The switches of a run are the troubled cells of every Runge-Kutta stage, the
Lax-Friedrichs speeds (alpha_x, alpha_y) of every stage and the time step of
every step.  With them fixed, the map from the initial moments to the final
ones is smooth almost everywhere (the absolute values in tau of Eq. (tao4) and
of Eq. (tao5) are its only kinks), and its vector-Jacobian product is the
adjoint the CUDA path computes.  Here that product is taken by PyTorch
autograd (CPU, float64) through a plain restatement of one stage in torch
operations: Step 4 (Step 1's formula per direction, characteristic fields of
the cell average for Euler), Step 5 (linear p0 at every Gauss point, HWENO at
the interface points of cells whose 3x3 stencil holds a troubled cell), the
Lax-Friedrichs fluxes, Eq. (ode2) and Eq. (RK).

Every reconstruction map is read off the C oracle, which derives it from the
moment conditions: candidate values at the Gauss points are linear in the 19
data and the smoothness indicators are quadratic forms in them, so evaluating
the C oracle's candidates on unit data (and on sums of two unit data, for the
quadratic forms) gives their matrices exactly up to rounding.  The switches
come from the C oracle's own forward run (`record`), and `frozen_step` (the C
oracle with the troubled cells given) is the forward map the finite-difference
checks differentiate.  Periodic boundaries and square cells only.
"""

import functools

import numpy as np
import torch

from . import oracle as O

_MOM = [1, 3, 4, 5, 7]                      # cells 2, 4, 5, 6, 8 (Fig. 1), 0-based
_OFF = [(di, dj) for dj in (-1, 0, 1) for di in (-1, 0, 1)]  # cells 1..9: (di, dj)
_RK = [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]  # Eq. (RK): u0 and stage weights
_G = 3                                      # ghost layers of the extended grid


def _gauss(ng):
    """Gauss-Legendre points and weights on [-1/2, 1/2] (weights sum to 1)."""
    x, w = np.polynomial.legendre.leggauss(ng)
    return 0.5 * x, 0.5 * w


@functools.lru_cache(maxsize=None)
def recon_tables(ng):
    """V [5][np][19]: candidate n at point p; B [5][19][19]: beta_n = d^T B_n d."""
    nd = 19
    npt = 4 * ng + ng * ng

    def cand(d):
        ub = np.array(d[:9], dtype=np.float64)
        vb = np.zeros(9)
        wb = np.zeros(9)
        vb[_MOM] = d[9:14]
        wb[_MOM] = d[14:19]
        return O.recon_candidates2d(ub, vb, wb, ng)

    V = np.zeros((5, npt, nd))
    bdiag = np.zeros((5, nd))
    for k in range(nd):
        e = np.zeros(nd)
        e[k] = 1.0
        val, beta = cand(e)
        V[:, :, k] = val
        bdiag[:, k] = beta
    B = np.zeros((5, nd, nd))
    for k in range(nd):
        B[:, k, k] = bdiag[:, k]
        for m in range(k + 1, nd):
            e = np.zeros(nd)
            e[k] = e[m] = 1.0
            _, beta = cand(e)
            B[:, k, m] = B[:, m, k] = 0.5 * (beta - bdiag[:, k] - bdiag[:, m])
    return torch.from_numpy(V), torch.from_numpy(B)


@functools.lru_cache(maxsize=None)
def limiter_tables():
    """Step 1 on data (u_m, u_0, u_p, v_m, v_p): q = Q d, beta_n = d^T B_n d."""
    def cand(d):
        return O.limiter_candidates1d(d[:3], d[3], d[4])
    Q = np.zeros((3, 5))
    bdiag = np.zeros((3, 5))
    for k in range(5):
        e = np.zeros(5)
        e[k] = 1.0
        q, beta = cand(e)
        Q[:, k] = q
        bdiag[:, k] = beta
    B = np.zeros((3, 5, 5))
    for k in range(5):
        B[:, k, k] = bdiag[:, k]
        for m in range(k + 1, 5):
            e = np.zeros(5)
            e[k] = e[m] = 1.0
            _, beta = cand(e)
            B[:, k, m] = B[:, m, k] = 0.5 * (beta - bdiag[:, k] - bdiag[:, m])
    return torch.from_numpy(Q), torch.from_numpy(B)


def _combine(gam, eps, beta, val, tau_scale):
    """Weights (99) with tau = (tau_scale sum_n |beta_0 - beta_n|)^2 and the
    combination omega_0 (v_0/gamma_0 - sum gamma_n/gamma_0 v_n) + sum omega_n v_n.
    beta: [N, ...], val: [N, ...] (broadcast)."""
    s = tau_scale * sum(torch.abs(beta[0] - beta[n]) for n in range(1, beta.shape[0]))
    tau = s * s
    wbar = [gam[n] * (1.0 + tau / (beta[n] + eps)) for n in range(beta.shape[0])]
    tot = sum(wbar)
    big = val[0] / gam[0]
    for n in range(1, beta.shape[0]):
        big = big - gam[n] / gam[0] * val[n]
    out = wbar[0] / tot * big
    for n in range(1, beta.shape[0]):
        out = out + wbar[n] / tot * val[n]
    return out


def euler_flux(g, U, direction):
    """Euler flux f (direction 0) or g (1) of U = (rho, m, n, E) [4, ...]."""
    rho, m, n, E = U[0], U[1], U[2], U[3]
    p = (g - 1.0) * (E - 0.5 * (m * m + n * n) / rho)
    vn = (m if direction == 0 else n) / rho
    return torch.stack([rho * vn, m * vn + (p if direction == 0 else 0.0),
                        n * vn + (p if direction == 1 else 0.0), vn * (E + p)])


def euler_eigen(g, U, direction):
    """Right (columns) and left (rows) eigenvectors of the x- or y-Jacobian at
    U [4, ...], eigenvalues ordered v - c, v, v, v + c (v the normal velocity)."""
    rho = U[0]
    mu, nu = U[1] / rho, U[2] / rho
    q2 = mu * mu + nu * nu
    p = (g - 1.0) * (U[3] - 0.5 * rho * q2)
    c = torch.sqrt(g * p / rho)
    H = (U[3] + p) / rho
    one, zero = torch.ones_like(rho), torch.zeros_like(rho)
    vn = mu if direction == 0 else nu
    if direction == 0:
        Rc = [[one, mu - c, nu, H - mu * c],
              [one, mu, nu, 0.5 * q2],
              [zero, zero, one, nu],
              [one, mu + c, nu, H + mu * c]]
    else:
        Rc = [[one, mu, nu - c, H - nu * c],
              [one, mu, nu, 0.5 * q2],
              [zero, one, zero, mu],
              [one, mu, nu + c, H + nu * c]]
    R = torch.stack([torch.stack(col) for col in Rc], dim=1)  # R[c][f]
    # left eigenvectors: the inverse of R (solved, not typed in)
    perm = list(range(2, R.dim())) + [0, 1]
    Rt = R.permute(*perm)
    Lt = torch.linalg.inv(Rt)
    inv_perm = [R.dim() - 2, R.dim() - 1] + list(range(R.dim() - 2))
    return R, Lt.permute(*inv_perm)


def _flux(system, g, U, direction):
    if system == O.BURGERS:
        return 0.5 * U * U
    return euler_flux(g, U, direction)


class Stage2D:
    """One evaluation of the operator of Eq. (ode2) with Step 4 and Step 5,
    troubled cells and (alpha_x, alpha_y) given, in torch float64."""

    def __init__(self, cfg):
        if cfg.bc != O.BC_PERIODIC:
            raise ValueError("the reference gradient is for periodic boundaries")
        self.cfg = cfg
        self.C = cfg.ncomp
        self.ng = 2 if cfg.n_gauss == 2 else 3
        self.dx = (cfg.x1 - cfg.x0) / cfg.nx
        self.dy = (cfg.y1 - cfg.y0) / cfg.ny
        if abs(self.dx - self.dy) > 1e-12 * self.dx:
            raise ValueError("square cells only")
        self.gam = [float(cfg.lin_w[k]) for k in range(5)]
        self.eps = float(cfg.eps)
        self.V, self.B = recon_tables(self.ng)
        self.Q1, self.B1 = limiter_tables()
        jj = torch.arange(-_G, cfg.ny + _G) % cfg.ny
        ii = torch.arange(-_G, cfg.nx + _G) % cfg.nx
        self.jj, self.ii = jj, ii

    # -- helpers on the extended grid [.., EY, EX]
    def _ext(self, a):
        return a[..., self.jj, :][..., :, self.ii]

    @staticmethod
    def _sh(a, di, dj, m):
        """a shifted by (di, dj), cropped by a margin m on each side."""
        EY, EX = a.shape[-2], a.shape[-1]
        return a[..., m + dj:EY - m + dj, m + di:EX - m + di]

    def _limit_scalar(self, um, u0, up, vm, vp):
        """Step 1's formula, elementwise."""
        D = torch.stack([um, u0, up, vm, vp])
        q = torch.einsum("nk,k...->n...", self.Q1, D)
        beta = torch.einsum("k...,nkl,l...->n...", D, self.B1, D)
        return _combine(self.gam[:3], self.eps, beta, q, 0.5)

    def limited(self, ue, fe):
        """Step 4 on the extended grid: (ub, vl, wl) [C, EY-2, EX-2] (margin 1)."""
        C = self.C
        ub, vb, wb = ue[:, 0], ue[:, 1], ue[:, 2]
        m = 1
        out = []
        for direction, mb in ((0, vb), (1, wb)):
            sx, sy = (1, 0) if direction == 0 else (0, 1)
            src = [self._sh(ub, -sx, -sy, m), self._sh(ub, 0, 0, m), self._sh(ub, sx, sy, m),
                   self._sh(mb, -sx, -sy, m), self._sh(mb, sx, sy, m)]
            if C == 1:
                lim = self._limit_scalar(*[s[0] for s in src])[None]
            else:
                g = self.cfg.gas_gamma
                R, L = euler_eigen(g, src[1], direction)
                W = [torch.einsum("fc...,c...->f...", L, s) for s in src]
                q = self._limit_scalar(*W)
                lim = torch.einsum("cf...,f...->c...", R, q)
            raw = self._sh(mb, 0, 0, m)
            out.append(torch.where(self._sh(fe, 0, 0, m).bool()[None], lim, raw))
        return self._sh(ub, 0, 0, m), out[0], out[1]

    def points(self, ue, fe):
        """Values at the 4 ng + ng^2 points of every cell of the extended grid
        with margin 2: [C, np, EY-4, EX-4]."""
        ng, C = self.ng, self.C
        nf = 4 * ng
        ub, vl, wl = self.limited(ue, fe)       # margin 1
        m = 1                                    # margin 2 relative to these
        d = [self._sh(ub, di, dj, m) for (di, dj) in _OFF]
        for k in _MOM:
            di, dj = _OFF[k]
            d.append(self._sh(vl, di, dj, m))
        for k in _MOM:
            di, dj = _OFF[k]
            d.append(self._sh(wl, di, dj, m))
        D = torch.stack(d, dim=1)                # [C, 19, H, W]
        lin = torch.einsum("pk,ckhw->cphw", self.V[0], D)
        f1 = self._sh(fe, 0, 0, 1).bool()
        hw = torch.zeros_like(self._sh(f1, 0, 0, 1))
        for (di, dj) in _OFF:
            hw = hw | self._sh(f1, di, dj, 1)
        if not bool(hw.any()):
            return lin
        Vf = self.V[:, :nf]
        if C == 1:
            val = torch.einsum("npk,ckhw->ncphw", Vf, D)
            beta = torch.einsum("ckhw,nkl,clhw->nchw", D, self.B, D)[:, :, None]
            faces = _combine(self.gam, self.eps, beta, val, 0.25)
        else:
            g = self.cfg.gas_gamma
            U = D[:, 4]
            parts = []
            for direction in (0, 1):
                R, L = euler_eigen(g, U, direction)
                E = torch.einsum("fchw,ckhw->fkhw", L, D)      # characteristic data
                val = torch.einsum("npk,fkhw->nfphw", Vf, E)
                beta = torch.einsum("fkhw,nkl,flhw->nfhw", E, self.B, E)[:, :, None]
                ch = _combine(self.gam, self.eps, beta, val, 0.25)   # [f, nf, H, W]
                full = torch.einsum("cfhw,fphw->cphw", R, ch)
                lo, hi = (0, 2 * ng) if direction == 0 else (2 * ng, 4 * ng)
                parts.append(full[:, lo:hi])
            faces = torch.cat(parts, dim=1)
        fpts = torch.where(hw[None, None], faces, lin[:, :nf])
        return torch.cat([fpts, lin[:, nf:]], dim=1)

    def rhs(self, u, flags, alpha_x, alpha_y):
        """L(u) [C, 3, ny, nx] and the limited state (ub, vl, wl) of the own cells."""
        ng, C = self.ng, self.C
        g = self.cfg.gas_gamma
        x, w = _gauss(ng)
        ue = self._ext(u)
        fe = self._ext(torch.as_tensor(flags, dtype=torch.uint8))
        P = self.points(ue, fe)                  # margin 2 -> own cells at margin 1
        me = self._sh(P, 0, 0, 1)
        ml, mr = self._sh(P, -1, 0, 1), self._sh(P, 1, 0, 1)
        mb, mt = self._sh(P, 0, -1, 1), self._sh(P, 0, 1, 1)
        hax, hay = 0.5 * alpha_x, 0.5 * alpha_y

        def lf(a, b, direction, h):
            return 0.5 * (_flux(self.cfg.system, g, a, direction)
                          + _flux(self.cfg.system, g, b, direction)) - h * (b - a)

        sfx = sfs = sfxe = sgy = sgs = sgyx = 0.0
        for k in range(ng):
            FL = lf(ml[:, ng + k], me[:, k], 0, hax)
            FR = lf(me[:, ng + k], mr[:, k], 0, hax)
            GB = lf(mb[:, 3 * ng + k], me[:, 2 * ng + k], 1, hay)
            GT = lf(me[:, 3 * ng + k], mt[:, 2 * ng + k], 1, hay)
            sfx = sfx + w[k] * (FR - FL)
            sfs = sfs + w[k] * (FL + FR)
            sfxe = sfxe + w[k] * x[k] * (FR - FL)
            sgy = sgy + w[k] * (GT - GB)
            sgs = sgs + w[k] * (GB + GT)
            sgyx = sgyx + w[k] * x[k] * (GT - GB)
        Fv = Gv = 0.0
        for l in range(ng):
            for k in range(ng):
                U = me[:, 4 * ng + l * ng + k]
                Fv = Fv + w[k] * w[l] * _flux(self.cfg.system, g, U, 0)
                Gv = Gv + w[k] * w[l] * _flux(self.cfg.system, g, U, 1)
        dx, dy = self.dx, self.dy
        L0 = -sfx / dx - sgy / dy
        L1 = -sfs / (2.0 * dx) + Fv / dx - sgyx / dy
        L2 = -sfxe / dx - sgs / (2.0 * dy) + Gv / dy
        ub, vl, wl = self.limited(ue, fe)
        lim = torch.stack([self._sh(ub, 0, 0, 2), self._sh(vl, 0, 0, 2),
                           self._sh(wl, 0, 0, 2)], dim=1)
        return torch.stack([L0, L1, L2], dim=1), lim

    def step(self, u, sw):
        """One step of Eq. (RK) with the switches sw = (flags[3], alphas[3], dt)."""
        flags, alphas, dt = sw
        W0 = None
        uk = u
        for s in range(3):
            L, lim = self.rhs(uk, flags[s], *alphas[s])
            if s == 0:
                W0 = lim
            a, b = _RK[s]
            uk = b * lim + b * dt * L if s == 0 else a * W0 + b * lim + b * dt * L
        return uk


# ------------------------------------------------------------ C-oracle side

def rhs_frozen(cfg, u, alpha_x, alpha_y, flags):
    """The C oracle's operator with the troubled cells given: (rhs, ulim)."""
    import ctypes
    u = O._state2d(cfg, u)
    rhs = np.empty_like(u)
    ulim = np.empty_like(u)
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    st = O.lib().hwo2d_rhs_fx(ctypes.byref(cfg), O._p(u), alpha_x, alpha_y,
                              fl.ctypes.data_as(O._PU8), O._p(rhs), O._p(ulim), None, None, None)
    if st != 0:
        raise FloatingPointError("oracle rhs2d_fx status %d" % st)
    return rhs, ulim


def frozen_step(cfg, u, sw):
    """One step of Eq. (RK) by the C oracle with the switches sw held fixed
    (the map the adjoint differentiates), combined in the order hwo2d_step uses."""
    flags, alphas, dt = sw
    L, W0 = rhs_frozen(cfg, u, *alphas[0], flags[0])
    uk = W0 + dt * L
    L, Wk = rhs_frozen(cfg, uk, *alphas[1], flags[1])
    uk = 0.75 * W0 + 0.25 * Wk + (0.25 * dt) * L
    L, Wk = rhs_frozen(cfg, uk, *alphas[2], flags[2])
    return (1.0 / 3.0) * W0 + (2.0 / 3.0) * Wk + ((2.0 / 3.0) * dt) * L


def record(cfg, u, nsteps, cfl):
    """The C oracle's own run (Eq. (RK), alpha per stage, dt per step from u^n)
    with its switches: returns (final state, [(flags[3], alphas[3], dt)])."""
    import ctypes
    u = O._state2d(cfg, u).copy()
    tape = []
    for _ in range(nsteps):
        dt = O.lib().hwo2d_dt(ctypes.byref(cfg), O._p(u), cfl, 0.0, -1.0)
        flags, alphas = [], []
        uk = u
        for s in range(3):
            ax, ay = O.alpha2d(cfg, uk)
            _, _, fl, _ = O.rhs2d(cfg, uk, ax, ay)
            flags.append(fl.copy())
            alphas.append((ax, ay))
            L, Wk = rhs_frozen(cfg, uk, ax, ay, fl)
            if s == 0:
                W0 = Wk
                uk = W0 + dt * L
            elif s == 1:
                uk = 0.75 * W0 + 0.25 * Wk + (0.25 * dt) * L
            else:
                uk = (1.0 / 3.0) * W0 + (2.0 / 3.0) * Wk + ((2.0 / 3.0) * dt) * L
        u = uk
        tape.append((flags, alphas, dt))
    return u, tape


def gradient(cfg, u0, tape, grad_out):
    """d<grad_out, u_N>/d u_0 through the frozen steps of tape (autograd)."""
    st = Stage2D(cfg)
    u = torch.tensor(np.asarray(u0, dtype=np.float64), requires_grad=True)
    x = u
    for sw in tape:
        x = st.step(x, sw)
    (x * torch.as_tensor(np.asarray(grad_out, dtype=np.float64))).sum().backward()
    return u.grad.numpy().copy(), x.detach().numpy().copy()


def rhs_vjp(cfg, u, flags, alpha_x, alpha_y, lam):
    """(dL/du)^T lam at u with the troubled cells and alphas fixed, where L
    includes Step 4 (the derivative of L(Lim(u)) with respect to the raw u)."""
    st = Stage2D(cfg)
    x = torch.tensor(np.asarray(u, dtype=np.float64), requires_grad=True)
    L, _ = st.rhs(x, flags, alpha_x, alpha_y)
    (L * torch.as_tensor(np.asarray(lam, dtype=np.float64))).sum().backward()
    return x.grad.numpy().copy(), L.detach().numpy().copy()
