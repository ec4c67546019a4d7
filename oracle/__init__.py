"""ORACLE -- test infrastructure only.

A plain FP64 CPU implementation of the hybrid Hermite WENO scheme with
artificial linear weights (Zhao & Qiu, arXiv:2002.08816, Sec. 2), written in C
(``hwo_*.c``) and loaded through ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package; the CUDA path in ``paper_2002_08816_gb300`` never does, and shares no
code with it.
"""

from .oracle import (  # noqa: F401
    BC_OUTFLOW,
    BC_PERIODIC,
    BC_REFLECTIVE,
    BURGERS,
    EULER,
    TROUBLED_ALL,
    TROUBLED_HYBRID,
    TROUBLED_NONE,
    Cfg1D,
    Cfg2D,
    build,
    lib,
)
