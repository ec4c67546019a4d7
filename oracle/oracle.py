"""ORACLE -- test infrastructure only: ctypes binding of the C oracle.

Functions mirror ``hweno_oracle.h``.  Arrays are float64 numpy arrays in the
structure-of-arrays layout the header documents.
"""

import ctypes
import glob
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libhweno_oracle.so")
# the same sources built with OpenMP: the per-cell loops run on all cores,
# the arithmetic of every cell unchanged
_LIB_OMP_PATH = os.path.join(_HERE, "libhweno_oracle_omp.so")
# the same sources compiled as C++ with a counting scalar (opcount.cpp)
_LIB_OPC_PATH = os.path.join(_HERE, "libhweno_oracle_opcount.so")

BURGERS, EULER = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_REFLECTIVE = 0, 1, 2
TROUBLED_HYBRID, TROUBLED_ALL, TROUBLED_NONE = 0, 1, 2

_D = ctypes.c_double
_I = ctypes.c_int
_PD = ctypes.POINTER(ctypes.c_double)
_PU8 = ctypes.POINTER(ctypes.c_uint8)
_PL = ctypes.POINTER(ctypes.c_long)


class Cfg1D(ctypes.Structure):
    _fields_ = [
        ("system", _I), ("nx", _I), ("x0", _D), ("x1", _D), ("bc", _I),
        ("gas_gamma", _D), ("lin_w", _D * 3), ("eps", _D),
        ("kxrcf_threshold", _D), ("troubled_mode", _I), ("limit_in_place", _I),
        ("char_state", _I),
    ]

    @classmethod
    def make(cls, system, nx, x0, x1, bc, lin_w=(0.98, 0.01, 0.01),
             gas_gamma=1.4, eps=1e-6, threshold=1.0,
             troubled_mode=TROUBLED_HYBRID, limit_in_place=1, char_state=0):
        c = cls()
        c.system, c.nx, c.x0, c.x1, c.bc = system, nx, x0, x1, bc
        c.gas_gamma = gas_gamma
        for k in range(3):
            c.lin_w[k] = lin_w[k]
        c.eps, c.kxrcf_threshold = eps, threshold
        c.troubled_mode, c.limit_in_place = troubled_mode, limit_in_place
        c.char_state = char_state
        return c

    @property
    def ncomp(self):
        return 3 if self.system == EULER else 1


class Cfg2D(ctypes.Structure):
    _fields_ = [
        ("system", _I), ("nx", _I), ("ny", _I), ("x0", _D), ("x1", _D),
        ("y0", _D), ("y1", _D), ("bc", _I), ("gas_gamma", _D),
        ("lin_w", _D * 5), ("eps", _D), ("kxrcf_threshold", _D),
        ("troubled_mode", _I), ("limit_in_place", _I), ("n_gauss", _I), ("char_state", _I),
    ]

    @classmethod
    def make(cls, system, nx, ny, x0, x1, y0, y1, bc,
             lin_w=(0.96, 0.01, 0.01, 0.01, 0.01), gas_gamma=1.4, eps=1e-6,
             threshold=1.0, troubled_mode=TROUBLED_HYBRID, limit_in_place=1,
             n_gauss=3, char_state=0):
        c = cls()
        c.system, c.nx, c.ny = system, nx, ny
        c.x0, c.x1, c.y0, c.y1, c.bc = x0, x1, y0, y1, bc
        c.gas_gamma = gas_gamma
        for k in range(5):
            c.lin_w[k] = lin_w[k]
        c.eps, c.kxrcf_threshold = eps, threshold
        c.troubled_mode, c.limit_in_place, c.n_gauss = troubled_mode, limit_in_place, n_gauss
        c.char_state = char_state
        return c

    @property
    def ncomp(self):
        return 4 if self.system == EULER else 1


def _build_one(path, extra, force):
    srcs = sorted(glob.glob(os.path.join(_HERE, "*.c")))
    if not force and os.path.exists(path):
        newest = max(os.path.getmtime(p) for p in srcs + glob.glob(os.path.join(_HERE, "*.h")))
        if os.path.getmtime(path) >= newest:
            return path
    tmp = path + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared"] + extra + \
        ["-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _build_opcount(force):
    srcs = [os.path.join(_HERE, f) for f in ("opcount.cpp", "opcount_1d.cpp", "opcount_2d.cpp")]
    deps = srcs + sorted(glob.glob(os.path.join(_HERE, "*.c"))) + glob.glob(os.path.join(_HERE, "*.h"))
    if not force and os.path.exists(_LIB_OPC_PATH):
        if os.path.getmtime(_LIB_OPC_PATH) >= max(os.path.getmtime(p) for p in deps):
            return
    tmp = _LIB_OPC_PATH + ".tmp%d" % os.getpid()
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + _HERE,
                    "-o", tmp] + srcs, check=True)
    os.replace(tmp, _LIB_OPC_PATH)


def build(force=False):
    """Compile the C oracle with gcc (no FMA contraction, so x86 and Arm agree),
    plain and with OpenMP (the second build is skipped where gcc has none), and
    the op-counting build of the same sources with g++."""
    _build_one(_LIB_PATH, [], force)
    try:
        _build_one(_LIB_OMP_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass
    try:
        _build_opcount(force)
    except (subprocess.CalledProcessError, OSError):
        pass  # measurement only: lib_opcount() then fails, the oracle itself does not
    return _LIB_PATH


_lib = None
_lib_omp = None
_lib_opc = None


def lib_opcount():
    """The op-counting build: the oracle's functions, plus hwo_opcount_read /
    hwo_opcount_reset (counts of add/sub, mul, div, sqrt, pow)."""
    global _lib_opc
    if _lib_opc is None:
        build()
        if not os.path.exists(_LIB_OPC_PATH):
            raise OSError("the op-counting build of the oracle (g++) is not available")
        L = _setup(ctypes.CDLL(_LIB_OPC_PATH))
        L.hwo_opcount_read.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        L.hwo_opcount_read.restype = None
        L.hwo_opcount_reset.argtypes = []
        L.hwo_opcount_reset.restype = None
        _lib_opc = L
    return _lib_opc


def count_ops(call):
    """The floating-point operations [add/sub, mul, div, sqrt, pow] the
    op-counting build performs in call(L) (L: that library), after one
    untimed warm-up call that builds the oracle's coefficient tables."""
    L = lib_opcount()
    call(L)
    L.hwo_opcount_reset()
    call(L)
    out = (ctypes.c_ulonglong * 5)()
    L.hwo_opcount_read(out)
    return [int(v) for v in out]


def lib_omp():
    """The OpenMP build (None when it could not be built)."""
    global _lib_omp
    if _lib_omp is None:
        build()
        if not os.path.exists(_LIB_OMP_PATH):
            return None
        _lib_omp = _setup(ctypes.CDLL(_LIB_OMP_PATH))
    return _lib_omp


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _setup(ctypes.CDLL(_LIB_PATH))
    return _lib


def threads(n=0):
    """Threads of the OpenMP build: sets the count when n > 0, returns it."""
    L = lib_omp()
    return L.hwo_set_threads(int(n)) if L is not None else 1


def _setup(L):
    """Argument and result types of the exported functions."""
    P1 = ctypes.POINTER(Cfg1D)
    L.hwo1d_alpha.restype = _D
    L.hwo1d_alpha.argtypes = [P1, _PD]
    L.hwo1d_rhs.restype = _I
    L.hwo1d_rhs.argtypes = [P1, _PD, _D, _PD, _PD, _PU8, _PD]
    L.hwo1d_rhs_ex.restype = _I
    L.hwo1d_rhs_ex.argtypes = [P1, _PD, _D, _PD, _PD, _PU8, _PD, _PD]
    L.hwo1d_step.restype = _I
    L.hwo1d_step.argtypes = [P1, _PD, _D, _PL]
    L.hwo1d_dt.restype = _D
    L.hwo1d_dt.argtypes = [P1, _PD, _D, _D, _D]
    L.hwo1d_run.restype = _I
    L.hwo1d_run.argtypes = [P1, _PD, _I, _D, _D, _D, _D, _PD, _PD, _PL]
    L.hwo1d_limiter_candidates.restype = None
    L.hwo1d_limiter_candidates.argtypes = [_PD, _D, _D, _PD, _PD]
    L.hwo1d_limit_scalar.restype = _D
    L.hwo1d_limit_scalar.argtypes = [_PD, _D, _PD, _D, _D]
    L.hwo1d_recon_candidates.restype = None
    L.hwo1d_recon_candidates.argtypes = [_PD, _PD, _PD, _PD]
    L.hwo1d_recon_scalar.restype = None
    L.hwo1d_recon_scalar.argtypes = [_PD, _D, _PD, _PD, _I, _PD]
    L.hwo_euler1d_eigen.restype = None
    L.hwo_euler1d_eigen.argtypes = [_D, _PD, _PD, _PD]
    L.hwo_euler1d_flux.restype = None
    L.hwo_euler1d_flux.argtypes = [_D, _PD, _PD]
    if hasattr(L, "hwo2d_rhs"):
        P2 = ctypes.POINTER(Cfg2D)
        L.hwo2d_rhs.restype = _I
        L.hwo2d_rhs.argtypes = [P2, _PD, _D, _D, _PD, _PD, _PU8, _PD]
        L.hwo2d_rhs_ex.restype = _I
        L.hwo2d_rhs_ex.argtypes = [P2, _PD, _D, _D, _PD, _PD, _PU8, _PD, _PD]
        L.hwo2d_rhs_fx.restype = _I
        L.hwo2d_rhs_fx.argtypes = [P2, _PD, _D, _D, _PU8, _PD, _PD, _PU8, _PD, _PD]
        L.hwo2d_alpha.restype = None
        L.hwo2d_alpha.argtypes = [P2, _PD, _PD, _PD]
        L.hwo2d_dt.restype = _D
        L.hwo2d_dt.argtypes = [P2, _PD, _D, _D, _D]
        L.hwo2d_step.restype = _I
        L.hwo2d_step.argtypes = [P2, _PD, _D, _PL]
        L.hwo2d_run.restype = _I
        L.hwo2d_run.argtypes = [P2, _PD, _I, _D, _D, _D, _D, _PD, _PD, _PL]
        L.hwo2d_recon_candidates.restype = _I
        L.hwo2d_recon_candidates.argtypes = [_PD, _PD, _PD, _I, _PD, _PD]
        L.hwo2d_linear_weights.restype = _I
        L.hwo2d_linear_weights.argtypes = [_I, _PD]
        L.hwo2d_p0_coeffs.restype = None
        L.hwo2d_p0_coeffs.argtypes = [_PD, _PD]
        L.hwo2d_quad_coeffs.restype = None
        L.hwo2d_quad_coeffs.argtypes = [_I, _PD, _PD]
        L.hwo2d_beta_of_coeffs.restype = _D
        L.hwo2d_beta_of_coeffs.argtypes = [_I, _PD, _D]
        L.hwo_euler2d_flux.restype = None
        L.hwo_euler2d_flux.argtypes = [_D, _PD, _I, _PD]
        L.hwo_euler2d_eigen.restype = None
        L.hwo_euler2d_eigen.argtypes = [_D, _PD, _I, _PD, _PD]
    L.hwo_set_threads.restype = _I
    L.hwo_set_threads.argtypes = [_I]
    return L


def _p(a):
    return a.ctypes.data_as(_PD)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _state1d(cfg, u):
    u = _f64(u)
    if u.size != cfg.ncomp * 2 * cfg.nx:
        raise ValueError("state of %d values does not match the 1D configuration" % u.size)
    return u


def _state2d(cfg, u):
    u = _f64(u)
    if u.size != cfg.ncomp * 3 * cfg.nx * cfg.ny:
        raise ValueError("state of %d values does not match the 2D configuration" % u.size)
    return u


# ----------------------------------------------------------------------------- 1D

def alpha1d(cfg, u):
    u = _state1d(cfg, u)
    return lib().hwo1d_alpha(ctypes.byref(cfg), _p(u))


def rhs1d(cfg, u, alpha=-1.0, faces=False):
    """One evaluation of Eq. (odeH).  Returns (rhs, ulim, flags, indicator),
    plus the interface values [C][2][nx] (u^+_{i-1/2}, u^-_{i+1/2}) if faces."""
    u = _state1d(cfg, u)
    rhs = np.empty_like(u)
    ulim = np.empty_like(u)
    fc = np.empty_like(u)
    flags = np.zeros(cfg.nx, dtype=np.uint8)
    ind = np.zeros(cfg.nx, dtype=np.float64)
    st = lib().hwo1d_rhs_ex(ctypes.byref(cfg), _p(u), alpha, _p(rhs), _p(ulim),
                            flags.ctypes.data_as(_PU8), _p(ind), _p(fc))
    if st != 0:
        raise FloatingPointError("oracle rhs1d status %d" % st)
    if faces:
        return rhs, ulim, flags, ind, fc
    return rhs, ulim, flags, ind


def dt1d(cfg, u, cfl, t=0.0, t_final=-1.0):
    u = _state1d(cfg, u)
    return lib().hwo1d_dt(ctypes.byref(cfg), _p(u), cfl, t, t_final)


def step1d(cfg, u, dt):
    """One SSP-RK3 step with the given dt; returns (u_new, troubled count)."""
    u = _state1d(cfg, u).copy()
    nt = ctypes.c_long(0)
    st = lib().hwo1d_step(ctypes.byref(cfg), _p(u), dt, ctypes.byref(nt))
    if st != 0:
        raise FloatingPointError("oracle step1d status %d" % st)
    return u, nt.value


def run1d(cfg, u, nsteps=-1, cfl=0.6, t0=0.0, t_final=-1.0, dt_fixed=-1.0,
          lin_w_per_step=None, omp=False):
    """Repeated SSP-RK3 steps; returns (u, t, troubled cell-stage count).
    omp: run the OpenMP build (same results, all cores; see threads())."""
    u = _state1d(cfg, u).copy()
    t = ctypes.c_double(0.0)
    nt = ctypes.c_long(0)
    lw = None
    if lin_w_per_step is not None:
        lw_arr = _f64(lin_w_per_step)
        assert nsteps >= 0 and lw_arr.size >= 3 * nsteps
        lw = _p(lw_arr)
    L = lib_omp() if omp else lib()
    st = (L or lib()).hwo1d_run(ctypes.byref(cfg), _p(u), nsteps, cfl, t0, t_final,
                                dt_fixed, lw, ctypes.byref(t), ctypes.byref(nt))
    if st != 0:
        raise FloatingPointError("oracle run1d status %d" % st)
    return u, t.value, nt.value


def limiter_candidates1d(ub3, v_m1, v_p1):
    ub3 = _f64(ub3)
    q = np.zeros(3)
    beta = np.zeros(3)
    lib().hwo1d_limiter_candidates(_p(ub3), v_m1, v_p1, _p(q), _p(beta))
    return q, beta


def limit_scalar1d(gam, eps, ub3, v_m1, v_p1):
    gam = _f64(gam)
    ub3 = _f64(ub3)
    return lib().hwo1d_limit_scalar(_p(gam), eps, _p(ub3), v_m1, v_p1)


def recon_candidates1d(ub3, vb3):
    ub3, vb3 = _f64(ub3), _f64(vb3)
    val = np.zeros(12)
    beta = np.zeros(3)
    lib().hwo1d_recon_candidates(_p(ub3), _p(vb3), _p(val), _p(beta))
    return val.reshape(3, 4), beta


def recon_scalar1d(gam, eps, ub3, vb3, hweno):
    gam, ub3, vb3 = _f64(gam), _f64(ub3), _f64(vb3)
    out = np.zeros(4)
    lib().hwo1d_recon_scalar(_p(gam), eps, _p(ub3), _p(vb3), int(hweno), _p(out))
    return out


def euler1d_eigen(g, U):
    U = _f64(U)
    R = np.zeros(9)
    L = np.zeros(9)
    lib().hwo_euler1d_eigen(g, _p(U), _p(R), _p(L))
    return R.reshape(3, 3), L.reshape(3, 3)


def euler1d_flux(g, U):
    U = _f64(U)
    F = np.zeros(3)
    lib().hwo_euler1d_flux(g, _p(U), _p(F))
    return F


# ----------------------------------------------------------------------------- 2D

# monomials xi^a eta^b, a + b <= 4, by total degree then descending a
MONO2D = [(a, d - a) for d in range(5) for a in range(d, -1, -1)]


def alpha2d(cfg, u):
    u = _state2d(cfg, u)
    ax, ay = ctypes.c_double(), ctypes.c_double()
    lib().hwo2d_alpha(ctypes.byref(cfg), _p(u), ctypes.byref(ax), ctypes.byref(ay))
    return ax.value, ay.value


def rhs2d(cfg, u, alpha_x=-1.0, alpha_y=-1.0, points=False):
    """One evaluation of Eq. (ode2).  Returns (rhs, ulim, flags, indicator),
    plus the reconstructed point values [C][np][ny][nx] if points."""
    u = _state2d(cfg, u)
    rhs = np.empty_like(u)
    ulim = np.empty_like(u)
    flags = np.zeros((cfg.ny, cfg.nx), dtype=np.uint8)
    ind = np.zeros((cfg.ny, cfg.nx), dtype=np.float64)
    ng = 2 if cfg.n_gauss == 2 else 3
    pts = np.zeros((u.shape[0], 4 * ng + ng * ng, cfg.ny, cfg.nx))
    st = lib().hwo2d_rhs_ex(ctypes.byref(cfg), _p(u), alpha_x, alpha_y, _p(rhs), _p(ulim),
                            flags.ctypes.data_as(_PU8), _p(ind), _p(pts))
    if st != 0:
        raise FloatingPointError("oracle rhs2d status %d" % st)
    if points:
        return rhs, ulim, flags, ind, pts
    return rhs, ulim, flags, ind


def step2d(cfg, u, dt):
    u = _state2d(cfg, u).copy()
    nt = ctypes.c_long(0)
    st = lib().hwo2d_step(ctypes.byref(cfg), _p(u), dt, ctypes.byref(nt))
    if st != 0:
        raise FloatingPointError("oracle step2d status %d" % st)
    return u, nt.value


def run2d(cfg, u, nsteps=-1, cfl=0.6, t0=0.0, t_final=-1.0, dt_fixed=-1.0,
          lin_w_per_step=None, omp=False):
    u = _state2d(cfg, u).copy()
    t = ctypes.c_double(0.0)
    nt = ctypes.c_long(0)
    lw = None
    if lin_w_per_step is not None:
        lw_arr = _f64(lin_w_per_step)
        assert nsteps >= 0 and lw_arr.size >= 5 * nsteps
        lw = _p(lw_arr)
    L = lib_omp() if omp else lib()
    st = (L or lib()).hwo2d_run(ctypes.byref(cfg), _p(u), nsteps, cfl, t0, t_final, dt_fixed,
                                lw, ctypes.byref(t), ctypes.byref(nt))
    if st != 0:
        raise FloatingPointError("oracle run2d status %d" % st)
    return u, t.value, nt.value


def recon_candidates2d(ub9, vb9, wb9, n_gauss=3):
    ub9, vb9, wb9 = _f64(ub9), _f64(vb9), _f64(wb9)
    np_ = 4 * n_gauss + n_gauss * n_gauss
    val = np.zeros(5 * 21)
    beta = np.zeros(5)
    lib().hwo2d_recon_candidates(_p(ub9), _p(vb9), _p(wb9), n_gauss, _p(val), _p(beta))
    return val[:5 * np_].reshape(5, np_), beta


def linear_weights2d(n_gauss=3):
    np_ = 4 * n_gauss + n_gauss * n_gauss
    W = np.zeros(21 * 19)
    lib().hwo2d_linear_weights(n_gauss, _p(W))
    return W[:np_ * 19].reshape(np_, 19)


def p0_coeffs2d(d19):
    d19 = _f64(d19)
    c = np.zeros(15)
    lib().hwo2d_p0_coeffs(_p(d19), _p(c))
    return c


def quad_coeffs2d(n, d19):
    d19 = _f64(d19)
    c = np.zeros(6)
    lib().hwo2d_quad_coeffs(int(n), _p(d19), _p(c))
    return c


def beta_of_coeffs2d(degree, c, ratio=1.0):
    c = _f64(c)
    return lib().hwo2d_beta_of_coeffs(int(degree), _p(c), ratio)


def euler2d_flux(g, U, direction):
    U = _f64(U)
    F = np.zeros(4)
    lib().hwo_euler2d_flux(g, _p(U), int(direction), _p(F))
    return F


def euler2d_eigen(g, U, direction):
    U = _f64(U)
    R = np.zeros(16)
    L = np.zeros(16)
    lib().hwo_euler2d_eigen(g, _p(U), int(direction), _p(R), _p(L))
    return R.reshape(4, 4), L.reshape(4, 4)
