"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/hweno.h declares, and rejects invalid configurations before touching
the GPU."""

import ctypes
import os
import re

import pytest

from paper_2002_08816_gb300 import build as B
from paper_2002_08816_gb300 import hweno as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return H.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hweno_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "hweno_create" in names and "hweno_rhs" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(H.EXPORTED) <= names


def _cfg(**kw):
    c = H.make_config(1, H.HWENO_EULER, 64)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("bad", [
    dict(nx=3), dict(dim=3), dict(system=7), dict(bc=5), dict(cfl=0.0), dict(eps=-1.0),
    dict(gas_gamma=1.0), dict(troubled_mode=9), dict(precision=4), dict(x1=0.0), dict(variant=4),
])
def test_invalid_configuration_is_rejected(lib, bad):
    h = ctypes.c_void_p()
    st = lib.hweno_create(ctypes.byref(_cfg(**bad)), None, ctypes.byref(h))
    assert st == H.HWENO_ERR_ARG
    assert h.value is None
    assert len(H.hweno_last_error(None)) > 0


@pytest.mark.parametrize("args", [(0, 1, 0, 10), (2000, 1, 0, 10), (4, 0, 0, 10), (4, 1, -1, 10),
                                  (4, 1, 2000, 10), (4, 1, 0, 0)])
def test_barrier_self_test_rejects_bad_arguments_before_cuda(lib, args):
    assert lib.hweno_check_barrier(*args) == H.HWENO_ERR_ARG
    assert b"hweno_check_barrier" in lib.hweno_last_error(None)


def test_pair_precision_is_refused_for_batches(lib):
    """HWENO_FP32C (float-pair averages) is refused for batches before any
    CUDA call."""
    h = ctypes.c_void_p()
    c1 = H.make_config(1, H.HWENO_EULER, 64, precision=H.HWENO_FP32C)
    sizes = (ctypes.c_int * 2)(64, 80)
    assert lib.hweno_create_batch(ctypes.byref(c1), 2, sizes, None, ctypes.byref(h)) == H.HWENO_ERR_ARG
    assert h.value is None


def test_linear_weights_must_be_positive_and_sum_to_one(lib):
    for w in ((0.5, 0.5, 0.0), (0.98, 0.01, 0.02), (1.2, -0.1, -0.1)):
        c = _cfg()
        for k in range(3):
            c.lin_w[k] = w[k]
        h = ctypes.c_void_p()
        assert lib.hweno_create(ctypes.byref(c), None, ctypes.byref(h)) == H.HWENO_ERR_ARG
    assert "weights" in H.hweno_last_error(None)


def test_default_config_matches_the_paper(lib):
    c = H.hweno_default_config(1, H.HWENO_EULER)
    assert list(c.lin_w)[:3] == [0.98, 0.01, 0.01]
    assert c.cfl == 0.6 and c.eps == 1e-6 and c.gas_gamma == 1.4
    c2 = H.hweno_default_config(2, H.HWENO_EULER)
    assert list(c2.lin_w) == [0.96, 0.01, 0.01, 0.01, 0.01]


def test_fma_peak_rejects_bad_arguments_before_any_cuda_call(lib):
    out = ctypes.c_double(0.0)
    assert lib.hweno_fma_peak(0, 0, ctypes.byref(out)) == H.HWENO_ERR_ARG
    assert lib.hweno_fma_peak(1, (1 << 24) + 1, ctypes.byref(out)) == H.HWENO_ERR_ARG
    assert lib.hweno_fma_peak(0, 10, None) == H.HWENO_ERR_ARG
    assert lib.hweno_fma_peak(3, 10, ctypes.byref(out)) == H.HWENO_ERR_ARG
    assert lib.hweno_fma_peak(-1, 10, ctypes.byref(out)) == H.HWENO_ERR_ARG
