"""Test-side helpers: exact solutions of the paper's smooth tests and the
parser of the hand-transcribed golden formulas.  No scheme arithmetic here."""

import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def burgers_exact_1d(x, t, n_newton=100):
    """u = 0.5 + sin(pi (x - u t)) solved by Newton (smooth for t < 1/pi)."""
    u = 0.5 + np.sin(np.pi * x)
    for _ in range(n_newton):
        s = x - u * t
        g = u - (0.5 + np.sin(np.pi * s))
        dg = 1.0 + np.pi * t * np.cos(np.pi * s)
        u = u - g / dg
    return u


def burgers_entropy_1d(x, t, nxi=4001):
    """Entropy solution of v_t + v v_x = 0, v(x, 0) = 0.5 + sin(pi x) (period
    2), also after the shock forms: the Hopf-Lax formula v = (x - xi*)/t with
    xi* minimising U0(xi) + (x - xi)^2 / (2 t), U0(xi) = xi/2 + (1 - cos(pi xi))/pi
    the integral of the initial data (a grid search over one period of feet,
    then Newton on the minimiser's stationarity condition)."""
    x = np.asarray(x, dtype=np.float64)
    if t == 0.0:
        return 0.5 + np.sin(np.pi * x)
    xs = x.reshape(-1)
    lo = xs[:, None] - 1.5 * t - 1.0
    xi = lo + np.linspace(0.0, 1.0, nxi)[None, :] * (3.0 * t + 2.0)

    def F(z, xx):
        return z / 2.0 + (1.0 - np.cos(np.pi * z)) / np.pi + (xx - z) ** 2 / (2.0 * t)
    k = np.argmin(F(xi, xs[:, None]), axis=1)
    z = xi[np.arange(xs.size), k]
    for _ in range(30):  # F'(z) = v0(z) - (x - z)/t = 0, F'' = pi cos(pi z) + 1/t > 0 at a min
        g = 0.5 + np.sin(np.pi * z) - (xs - z) / t
        dg = np.pi * np.cos(np.pi * z) + 1.0 / t
        z = z - g / np.where(np.abs(dg) > 1e-12, dg, 1e-12)
    return ((xs - z) / t).reshape(x.shape)


def _coef(tok):
    """'p/q' -> (a, 0); 'A~B' -> (a, b) meaning a + b sqrt(5)."""
    if "~" in tok:
        a, b = tok.split("~")
        return float(Fraction(a)), float(Fraction(b))
    return float(Fraction(tok)), 0.0


def load_printed_1d():
    """Returns (lin, beta): lin[name] = (cite, coeffs[6]); beta[name] = (cite,
    [(w, coeffs[6]), ...])."""
    lin, beta = {}, {}
    cur = None
    r5 = np.sqrt(5.0)
    with open(os.path.join(GOLDEN, "hweno1d_printed.txt")) as fh:
        for raw in fh:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("lin "):
                name, cite, cs = [p.strip() for p in line[4:].split("|")]
                vals = [_coef(t) for t in cs.split()]
                lin[name] = (cite, np.array([a + b * r5 for a, b in vals]))
                cur = None
            elif line.startswith("beta "):
                name, cite = [p.strip() for p in line[5:].split("|")]
                beta[name] = (cite, [])
                cur = name
            elif line.startswith("sq "):
                w, cs = [p.strip() for p in line[3:].split("|")]
                beta[cur][1].append((float(Fraction(w)),
                                     np.array([_coef(t)[0] for t in cs.split()])))
    return lin, beta


def eval_beta(terms, d):
    return sum(w * float(c @ d) ** 2 for w, c in terms)
