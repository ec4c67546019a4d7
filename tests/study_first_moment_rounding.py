"""Which FP32 rounding limits the first moments of the shocked 1D workload?

A study on the FP64 oracle (not collected by pytest; run by hand, about 2
minutes per variant on 8 host cores):

  python tests/study_first_moment_rounding.py [--steps 2000] [--threads 8]

The 65536-cell two-state 1D Euler workload (seed 20250, outflow, CFL 0.5,
input rounded to FP32) is advanced with the oracle's right-hand side
(Eq. (odeH)) and the SSP-RK3 combination of Eq. (RK) written out here in
FP64, with one of these roundings to FP32 applied at every stage:

  store_avg   the cell averages of every stage output (first moments exact);
  store_both  averages and first moments of every stage output (FP32
              storage with exact arithmetic);
  eval_input  the right-hand side evaluated from the FP32-rounded stage
              input while the state itself is kept in FP64.

Each run is compared with the unrounded FP64 run: relative L1 per
component, averages and first moments.  The first moments' right-hand side
reacts to a perturbation of the averages with a factor 1/dx, so a
rounding-level change of the averages anywhere in the path shows in the
first moments at ~1e-2 relative after the 2000 shocked steps; none of these
splits brings them near 1e-4, which needs the whole path in FP64.
"""

import argparse
import ctypes
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import oracle as O  # noqa: E402
from paper_2002_08816_gb300 import workloads as W  # noqa: E402

NX, CFL, SEED = 65536, 0.5, 20250


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--variants", default="store_avg,store_both,eval_input")
    args = ap.parse_args()
    L = O.lib_omp() or O.lib()
    O.threads(args.threads)
    cfg = O.Cfg1D.make(O.EULER, NX, 0.0, 1.0, O.BC_OUTFLOW)
    dx = 1.0 / NX
    u0 = W.euler_two_state_1d(NX, seed=SEED).astype(np.float32).astype(np.float64)
    u0 = u0.reshape(3, 2, NX)
    rhs = np.empty(u0.size)
    ulim = np.empty(u0.size)
    flags = np.zeros(NX, np.uint8)
    ind = np.zeros(NX)

    def r32(a):
        return a.astype(np.float32).astype(np.float64)

    def Lop(u, variant):
        """Eq. (odeH) of the stage input and the input with Step 1's modified
        first moments on the troubled cells (what Eq. (RK) combines)."""
        x = np.ascontiguousarray((r32(u) if variant == "eval_input" else u).reshape(-1))
        st = L.hwo1d_rhs(ctypes.byref(cfg), O._p(x), -1.0, O._p(rhs), O._p(ulim),
                         flags.ctypes.data_as(O._PU8), O._p(ind))
        if st != 0:
            raise FloatingPointError("oracle rhs status %d" % st)
        base = u.copy()
        t = flags != 0
        base[:, 1, t] = ulim.reshape(3, 2, NX)[:, 1, t]
        return rhs.reshape(3, 2, NX).copy(), base

    def store(u, variant):
        if variant == "store_avg":
            u = u.copy()
            u[:, 0] = r32(u[:, 0])
        elif variant == "store_both":
            u = r32(u)
        return u

    def run(variant):
        u = u0.copy()
        for _ in range(args.steps):
            alpha = L.hwo1d_alpha(ctypes.byref(cfg), O._p(np.ascontiguousarray(u.reshape(-1))))
            dt = CFL * dx / alpha
            L0, b0 = Lop(u, variant)
            u1 = store(b0 + dt * L0, variant)
            L1, b1 = Lop(u1, variant)
            u2 = store(0.75 * b0 + 0.25 * b1 + 0.25 * dt * L1, variant)
            L2, b2 = Lop(u2, variant)
            u = store(b0 / 3.0 + (2.0 / 3.0) * b2 + (2.0 / 3.0) * dt * L2, variant)
        return u

    t0 = time.time()
    ref = run("fp64")
    print("fp64 reference: %.1f s" % (time.time() - t0), flush=True)
    if args.steps > 0:  # the loop above is the oracle's own step (Eq. (RK)) up to rounding
        cmp, _, _ = O.run1d(cfg, u0.reshape(-1), nsteps=args.steps, cfl=CFL,
                            omp=O.lib_omp() is not None)
        print("fp64 loop against the oracle's run: max |diff| %.2e" % np.abs(
            cmp.reshape(ref.shape) - ref).max(), flush=True)
    for variant in args.variants.split(","):
        t0 = time.time()
        u = run(variant)
        err = np.abs(u - ref).sum(axis=2) / np.abs(ref).sum(axis=2)
        print("%-11s %6.1f s  averages rel L1 %s  first moments rel L1 %s" % (
            variant, time.time() - t0, " ".join("%.2e" % e for e in err[:, 0]),
            " ".join("%.2e" % e for e in err[:, 1])), flush=True)


if __name__ == "__main__":
    main()
