"""Short run of the 1D stage kernels for profilers (ncu).

  python -m paper_2002_08816_gb300.profile_stage [--nx 65536] [--rk-steps 10]
                                                  [--precision fp32|fp32c|fp64] [--system euler|burgers]
                                                  [--dim 1|2] [--n-gauss 2|3]
                                                  [--adjoint EVERY] [--threads 128|256|512]
                                                  [--persistent | --resident] [--batch N]
                                                  [--quadrants] [--lax-tiles]

Sets the seeded two-state 1D Euler state (or the Burgers sine wave; with
--dim 2 the nx x nx vortex-plus-modes 2D Euler state), runs the
requested number of Runge-Kutta steps through the C ABI (3 stage launches per
step after one alpha launch) and checks the status word.  With --adjoint
EVERY (2D) the steps are recorded with a checkpoint every EVERY steps and the
gradient of sum(rho^2) is taken (hweno_backward: recomputed stages, then two
adjoint kernels per stage).  With --batch N it runs N independent 1D Euler
instances in shared launches (hweno_create_batch).  --persistent and
--resident select the 1D launch kinds with one launch per run.  --quadrants
(2D) replaces the vortex by four constant quadrants drawn from the seed (shocks
along the quadrant lines: the troubled-cell paths); --lax-tiles (1D Euler)
replaces the two-state data by Lax's Riemann problem repeated every 800 cells
(10-14 % of the cell-stages troubled).
"""

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import numpy as np
    import torch

    from paper_2002_08816_gb300 import build as B
    from paper_2002_08816_gb300 import hweno as H
    from paper_2002_08816_gb300 import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=65536)
    ap.add_argument("--rk-steps", type=int, default=10)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32c", "fp64"],
                    help="fp32c: FP32 with float-pair averages (1D: the resident launch)")
    ap.add_argument("--system", default="euler", choices=["euler", "burgers"])
    ap.add_argument("--seed", type=int, default=20250)
    ap.add_argument("--dim", type=int, default=1, choices=[1, 2])
    ap.add_argument("--n-gauss", type=int, default=2, choices=[2, 3])
    ap.add_argument("--adjoint", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0, choices=[0, 128, 256, 512],
                    help="1D: threads per CTA (0: the default)")
    ap.add_argument("--persistent", action="store_true",
                    help="1D: one persistent launch with grid barriers instead of per-stage graphs")
    ap.add_argument("--resident", action="store_true",
                    help="1D FP32: one resident launch (tiles kept on chip) per run")
    ap.add_argument("--quadrants", action="store_true",
                    help="2D Euler: four constant quadrants drawn from the seed instead of the vortex")
    ap.add_argument("--lax-tiles", action="store_true",
                    help="1D Euler: Lax's problem repeated every 800 cells, periodic")
    ap.add_argument("--batch", type=int, default=0,
                    help="1D Euler: this many instances, cells log-uniform in [256, 16384], "
                         "two-state data (the batched workload's recipe, seed 77)")
    args = ap.parse_args()
    B.build()
    prec = {"fp32": H.HWENO_FP32, "fp32c": H.HWENO_FP32C, "fp64": H.HWENO_FP64}[args.precision]
    sdt = H.HWENO_FP64 if prec == H.HWENO_FP64 else H.HWENO_FP32  # the state's element type
    if args.dim == 2:
        # 2D Euler, nx x nx periodic on [0, 10]^2, vortex plus density modes
        if args.quadrants:
            u = W.euler_quadrants_2d(args.nx, args.nx, seed=args.seed)
        else:
            u = W.euler_vortex_modes_2d(args.nx, args.nx, seed=args.seed, npts=2)
        cfg = H.make_config(2, H.HWENO_EULER, args.nx, args.nx, x0=0.0, x1=10.0, y0=0.0,
                            y1=10.0, cfl=0.5, precision=prec, n_gauss=args.n_gauss)
    elif args.batch > 0:
        sizes = [int(v) for v in W.batch_sizes_1d(args.batch, seed=77)]
        u = np.concatenate([W.euler_two_state_1d(n, seed=77 + b).reshape(-1)
                            for b, n in enumerate(sizes)])
        cfg = H.make_config(1, H.HWENO_EULER, 4, x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW, cfl=0.5,
                            precision=prec)
    elif args.system == "euler" and args.lax_tiles:
        u = W.euler_lax_tiled_1d(args.nx)
        cfg = H.make_config(1, H.HWENO_EULER, args.nx, x0=0.0, x1=1.0, bc=H.HWENO_BC_PERIODIC, cfl=0.5,
                            precision=prec)
    elif args.system == "euler":
        u = W.euler_two_state_1d(args.nx, args.seed)
        cfg = H.make_config(1, H.HWENO_EULER, args.nx, x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW, cfl=0.5,
                            precision=prec)
    else:
        u = W.burgers_sine_1d(args.nx)
        cfg = H.make_config(1, H.HWENO_BURGERS, args.nx, x0=-1.0, x1=1.0, cfl=0.5, precision=prec)
    dt = torch.float64 if sdt == H.HWENO_FP64 else torch.float32
    dev = torch.from_numpy(u).to("cuda", dt).contiguous()
    if args.batch > 0:
        h = H.hweno_create_batch(cfg, sizes, torch.cuda.current_stream().cuda_stream)
    else:
        h = H.hweno_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        if (args.threads or args.persistent or args.resident) and args.dim == 1:
            resident = args.resident or prec == H.HWENO_FP32C  # fp32c: always resident
            H.hweno_set_execution(h, args.threads or 256,
                                  2 if resident else (1 if args.persistent else 0))
        H.hweno_set_state(h, dev.data_ptr(), sdt, True)
        if args.adjoint > 0:
            t = H.hweno_record(h, args.rk_steps, args.adjoint)
            out = torch.empty_like(dev)
            H.hweno_get_state(h, out.data_ptr(), sdt, True)
            seed = torch.zeros_like(dev)
            seed[0, 0] = 2.0 * out[0, 0]
            grad = torch.empty_like(dev)
            H.hweno_backward(h, seed.data_ptr(), grad.data_ptr(), sdt, True)
            print("gradient norm %.6g" % float(grad.double().norm()))
        else:
            t = H.hweno_step(h, args.rk_steps)
        st = H.hweno_stats(h)
    finally:
        H.hweno_destroy(h)
    print("t=%.6g steps=%d troubled cell-stages=%d" % (t, st["steps"], st["troubled"]))


if __name__ == "__main__":
    main()
