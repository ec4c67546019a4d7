"""Thin ctypes binding of libhweno.so (include/hweno.h), same names as the C ABI.

Argument marshalling only: every step of the scheme runs in the library's
CUDA kernels.  Device buffers are passed as integers (e.g. a torch tensor's
``data_ptr()``), streams as integers (``torch.cuda.current_stream().cuda_stream``).
Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhweno.so")

HWENO_OK, HWENO_ERR_ARG, HWENO_ERR_CUDA, HWENO_ERR_NONPHYSICAL, HWENO_ERR_TIMEOUT, \
    HWENO_ERR_STATE, HWENO_ERR_TOO_LARGE = range(7)
HWENO_NOALLOC_MAX_CELLS = 4194304
HWENO_BURGERS, HWENO_EULER = 0, 1
HWENO_BC_PERIODIC, HWENO_BC_OUTFLOW, HWENO_BC_REFLECTIVE = 0, 1, 2
HWENO_VARIANT_RAW_COMBINE = 1  # the RK combination uses the unmodified first moments
HWENO_VARIANT_MEAN_EIGEN = 2  # characteristic fields of each interface's mean state
HWENO_TROUBLED_HYBRID, HWENO_TROUBLED_ALL, HWENO_TROUBLED_NONE = 0, 1, 2
HWENO_FP32, HWENO_FP64, HWENO_FP32C = 0, 1, 2

_D, _I, _VP = ctypes.c_double, ctypes.c_int, ctypes.c_void_p

EXPORTED = ["hweno_default_config", "hweno_create", "hweno_set_state", "hweno_step",
            "hweno_rhs", "hweno_get_state", "hweno_stats", "hweno_destroy",
            "hweno_last_error", "hweno_rhs1d_noalloc", "hweno_create_batch",
            "hweno_batch_times", "hweno_check_barrier"]


class hweno_config(ctypes.Structure):
    _fields_ = [
        ("dim", _I), ("system", _I), ("nx", _I), ("ny", _I),
        ("x0", _D), ("x1", _D), ("y0", _D), ("y1", _D),
        ("bc", _I), ("gas_gamma", _D), ("lin_w", _D * 5), ("cfl", _D), ("eps", _D),
        ("kxrcf_threshold", _D), ("troubled_mode", _I), ("n_gauss", _I), ("precision", _I),
        ("variant", _I),
    ]


class HwenoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("hweno status %d: %s" % (status, msg))
        self.status = status


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhweno.so is not built (run __graft_entry__.build()); "
                              "this package has no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(hweno_config)
        L.hweno_default_config.restype = None
        L.hweno_default_config.argtypes = [P, _I, _I]
        L.hweno_create.restype = _I
        L.hweno_create.argtypes = [P, _VP, ctypes.POINTER(_VP)]
        L.hweno_set_state.restype = _I
        L.hweno_set_state.argtypes = [_VP, _VP, _I, _I]
        L.hweno_step.restype = _I
        L.hweno_step.argtypes = [_VP, _I, _D, ctypes.POINTER(_D)]
        L.hweno_rhs.restype = _I
        L.hweno_rhs.argtypes = [_VP, _VP, _VP, _VP, _VP]
        L.hweno_get_state.restype = _I
        L.hweno_get_state.argtypes = [_VP, _VP, _I, _I]
        L.hweno_stats.restype = _I
        L.hweno_stats.argtypes = [_VP, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.hweno_destroy.restype = None
        L.hweno_destroy.argtypes = [_VP]
        L.hweno_last_error.restype = ctypes.c_char_p
        L.hweno_last_error.argtypes = [_VP]
        L.hweno_create_batch.restype = _I
        L.hweno_create_batch.argtypes = [P, _I, ctypes.POINTER(_I), _VP, ctypes.POINTER(_VP)]
        L.hweno_batch_times.restype = _I
        L.hweno_batch_times.argtypes = [_VP, ctypes.POINTER(_D)]
        L.hweno_record.restype = _I
        L.hweno_record.argtypes = [_VP, _I, _I, _D, ctypes.POINTER(_D)]
        L.hweno_backward.restype = _I
        L.hweno_backward.argtypes = [_VP, _VP, _VP, _I, _I]
        L.hweno_rhs_vjp.restype = _I
        L.hweno_rhs_vjp.argtypes = [_VP, _VP, _VP, _D, _D, _VP, _VP]
        L.hweno_totals.restype = _I
        L.hweno_totals.argtypes = [_VP, ctypes.POINTER(_D)]
        L.hweno_set_execution.restype = _I
        L.hweno_set_execution.argtypes = [_VP, _I, _I]
        L.hweno_autotune.restype = _I
        L.hweno_autotune.argtypes = [_VP, _I, ctypes.POINTER(_I)]
        L.hweno_check_barrier.restype = _I
        L.hweno_check_barrier.argtypes = [_I, _I, _I, ctypes.c_uint]
        L.hweno_rhs1d_noalloc.restype = _I
        L.hweno_rhs1d_noalloc.argtypes = [P, _VP, _VP, _VP, _VP, _VP]
        L.hweno_fma_peak.restype = _I
        L.hweno_fma_peak.argtypes = [_I, _I, ctypes.POINTER(_D)]
        L.hweno_check_resident.restype = _I
        L.hweno_check_resident.argtypes = [_VP, _I, _I, ctypes.c_uint]
        _lib = L
    return _lib


def _check(st, h=None):
    if st != HWENO_OK:
        raise HwenoError(st, lib().hweno_last_error(h).decode())


def hweno_default_config(dim, system):
    cfg = hweno_config()
    lib().hweno_default_config(ctypes.byref(cfg), dim, system)
    return cfg


def hweno_create(cfg, stream=0):
    h = _VP()
    _check(lib().hweno_create(ctypes.byref(cfg), _VP(stream or None), ctypes.byref(h)))
    return h.value


def hweno_create_batch(cfg, nx_list, stream=0):
    n = len(nx_list)
    arr = (_I * n)(*[int(v) for v in nx_list])
    h = _VP()
    _check(lib().hweno_create_batch(ctypes.byref(cfg), n, arr, _VP(stream or None), ctypes.byref(h)))
    return h.value


def hweno_batch_times(h, n):
    t = (_D * n)()
    _check(lib().hweno_batch_times(h, t), h)
    return list(t)


def hweno_set_state(h, ptr, dtype, on_device):
    _check(lib().hweno_set_state(h, _VP(ptr), dtype, int(on_device)), h)


def hweno_step(h, nsteps, t_final=-1.0, wait=True):
    """Returns the time reached when wait, else None (asynchronous)."""
    if wait:
        t = _D()
        _check(lib().hweno_step(h, int(nsteps), float(t_final), ctypes.byref(t)), h)
        return t.value
    _check(lib().hweno_step(h, int(nsteps), float(t_final), None), h)
    return None


def hweno_rhs(h, in_ptr, out_ptr, flags_ptr=0, ulim_ptr=0):
    _check(lib().hweno_rhs(h, _VP(in_ptr), _VP(out_ptr), _VP(flags_ptr or None),
                           _VP(ulim_ptr or None)), h)


def hweno_rhs1d_noalloc(cfg, stream, in_ptr, out_ptr, flags_ptr=0, ulim_ptr=0):
    """Allocation-free 1D right-hand side; returns the raw status code (no
    handle, so no error text)."""
    return lib().hweno_rhs1d_noalloc(ctypes.byref(cfg), _VP(stream or None), _VP(in_ptr),
                                     _VP(out_ptr), _VP(flags_ptr or None), _VP(ulim_ptr or None))


def hweno_record(h, nsteps, checkpoint_every, t_final=-1.0):
    """Runs nsteps steps recording the tape for hweno_backward; returns t."""
    t = _D()
    _check(lib().hweno_record(h, int(nsteps), int(checkpoint_every), float(t_final),
                              ctypes.byref(t)), h)
    return t.value


def hweno_backward(h, grad_out_ptr, grad_in_ptr, dtype, on_device):
    _check(lib().hweno_backward(h, _VP(grad_out_ptr), _VP(grad_in_ptr), dtype, int(on_device)), h)


def hweno_rhs_vjp(h, in_ptr, flags_ptr, alpha_x, alpha_y, lam_ptr, grad_ptr):
    _check(lib().hweno_rhs_vjp(h, _VP(in_ptr), _VP(flags_ptr), float(alpha_x), float(alpha_y),
                               _VP(lam_ptr), _VP(grad_ptr)), h)


def hweno_autotune(h, nsteps_trial):
    """Returns (threads per CTA, launch kind) chosen for the 1D handle: 0
    per-stage graphs, 1 persistent, 2 resident."""
    out = (_I * 2)()
    _check(lib().hweno_autotune(h, int(nsteps_trial), out), h)
    return out[0], out[1]


def hweno_totals(h, count):
    """The count (= instances x components) conserved totals, FP64."""
    out = (_D * count)()
    _check(lib().hweno_totals(h, out), h)
    return list(out)


def hweno_check_barrier(ctas, meetings, missing, polls):
    """Self-test of the persistent launch's bounded grid barrier; returns the
    status code (HWENO_OK, or HWENO_ERR_TIMEOUT when a wait ran out) and raises
    HwenoError on other failures."""
    st = lib().hweno_check_barrier(int(ctas), int(meetings), int(missing), int(polls))
    if st not in (HWENO_OK, HWENO_ERR_TIMEOUT):
        raise HwenoError(st, lib().hweno_last_error(None).decode())
    return st


def hweno_fma_peak(kind, iters):
    """Measured FMA throughput of the current device, flops per second (kind:
    0 or False FP32, 1 or True FP64, 2 packed FP32)."""
    out = _D()
    _check(lib().hweno_fma_peak(int(kind), int(iters), ctypes.byref(out)))
    return out.value


def hweno_check_resident(h, nsteps, silent_cta, polls):
    """Self-test of the resident launch's bounded waits; returns the status
    code (HWENO_OK, or HWENO_ERR_TIMEOUT when a wait ran out) and raises
    HwenoError on other failures."""
    st = lib().hweno_check_resident(h, int(nsteps), int(silent_cta), int(polls))
    if st not in (HWENO_OK, HWENO_ERR_TIMEOUT):
        raise HwenoError(st, lib().hweno_last_error(h).decode())
    return st


def hweno_set_execution(h, threads, persistent):
    _check(lib().hweno_set_execution(h, int(threads), int(persistent)), h)


def hweno_get_state(h, ptr, dtype, on_device):
    _check(lib().hweno_get_state(h, _VP(ptr), dtype, int(on_device)), h)


def hweno_stats(h):
    t, dt = _D(), _D()
    steps, tr = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().hweno_stats(h, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(steps),
                             ctypes.byref(tr)), h)
    return {"t": t.value, "dt": dt.value, "steps": steps.value, "troubled": tr.value}


def hweno_destroy(h):
    if h:
        lib().hweno_destroy(h)


def hweno_last_error(h=None):
    return lib().hweno_last_error(h).decode()


def make_config(dim, system, nx, ny=0, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=HWENO_BC_PERIODIC,
                lin_w=None, cfl=0.6, precision=HWENO_FP32, troubled_mode=HWENO_TROUBLED_HYBRID,
                gas_gamma=1.4, eps=1e-6, threshold=1.0, n_gauss=3, variant=0):
    cfg = hweno_default_config(dim, system)
    cfg.nx, cfg.ny = nx, ny
    cfg.x0, cfg.x1, cfg.y0, cfg.y1 = x0, x1, y0, y1
    cfg.bc, cfg.cfl, cfg.precision, cfg.troubled_mode = bc, cfl, precision, troubled_mode
    cfg.gas_gamma, cfg.eps, cfg.kxrcf_threshold, cfg.n_gauss = gas_gamma, eps, threshold, n_gauss
    cfg.variant = variant
    if lin_w is not None:
        for k, v in enumerate(lin_w):
            cfg.lin_w[k] = v
    return cfg
