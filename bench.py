"""Benchmark of the hybrid HWENO time stepper on GB300.

Workload (one bench step): the seeded two-state 1D Euler problem, gamma 1.4,
65536 cells on [0, 1] with outflow ends, advanced 2000 third-order TVD
Runge-Kutta steps (6000 stages, 3.93e8 cell-stages) at CFL 0.5, FP32 bulk
arithmetic (the time itself accumulated in FP64).  The metric is cell-updates per second counted
per Runge-Kutta stage.  The FP64 path is timed on the same workload and
reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hweno|reference]

--impl reference times the FP64 C oracle on the host cores on a bounded
sample of the same workload.  Under torchrun each rank advances its own
seeded instance (no data-path collective): weak scaling.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = 65536
RK_STEPS = 2000
CFL = 0.5
SEED = 20250
METRIC = "cell-updates/s (x RK stages) of the hybrid HWENO step"
UNIT = "cell-stages/s"
# algorithmic bytes per cell-stage: stage 1 reads u^n and writes u^(1) (2S),
# stages 2 and 3 read u^n and u^(k) and write (3S); mean 8S/3 with
# S = 3 components x 2 moments x sizeof(real)
BYTES_PER_CELL_STAGE = {"fp32": 8 * 24 / 3, "fp64": 8 * 48 / 3}
# DRAM bytes (read + write) per stage from ncu captures of the current kernels,
# summarised under profiles/: 1D per-stage launches, the mean over the three
# stages at the bench's 65536 cells, cold L2; the 1D persistent launch, its
# bytes over its 6000 stages; 2D, a 2048^2 capture scaled by the cell count to
# 4096^2
TRAFFIC_1D_FP32 = {(128, "per-stage graphs"): (3188224 + 2304 + 1741568 + 768 + 3183104 + 768) / 3,
                   (256, "per-stage graphs"): (3181568 + 1608448 + 3181312) / 3,
                   (512, "per-stage graphs"): (3181568 + 1608448 + 3181312) / 3,
                   # one persistent launch of 2000 steps: the state stays in L2
                   (256, "persistent"): (2301696 + 280064) / 6000,
                   (128, "persistent"): (2735360 + 475904) / 6000}
# the batched workload (512 instances): DRAM bytes per stage launch, the mean
# over the three stages, cold L2
TRAFFIC_BATCH_FP32 = {(128, False): (97092096 + 26866432 + 49318144 + 46779904 + 97016064 + 24710400) / 3,
                      (256, False): (95641344 + 19350528 + 47903488 + 36089600 + 95667712 + 17846784) / 3}
TRAFFIC_2D_NG2 = 4 * (403427584 + 178328320 + 403399680 + 179353600) / 2
L2_FLUSH_BYTES = 512 << 20


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device="cuda"):
    """The slowest rank's time: an all-reduce MAX over the process group (one
    independent replica per rank, so this is the only collective); x itself
    when there is no group or one rank."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size, units_per_rank, seconds):
    """Whole-job throughput of weak-scaled replicas: every rank processes
    units_per_rank units, the job takes the slowest rank's seconds."""
    return world_size * units_per_rank / seconds


def workload(rank):
    from paper_2002_08816_gb300 import workloads as W
    return W.euler_two_state_1d(NX, seed=SEED + rank)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = float(f[2])
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                         "sw_power_cap"]
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_cpu_baseline(u0, budget_s=12.0, max_steps=400):
    """The FP64 C oracle as it stands, single-threaded, on the full 65536-cell
    state for as many RK steps as fit in about budget_s seconds."""
    from oracle import oracle as O
    cfg = O.Cfg1D.make(O.EULER, NX, 0.0, 1.0, O.BC_OUTFLOW)
    u = u0.copy()
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        u, _, _ = O.run1d(cfg, u, nsteps=5, cfl=CFL)
        steps += 5
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": NX * 3 * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d of the %d RK steps of the 65536-cell workload, FP64, 1 thread, %.1f s"
                      % (steps, RK_STEPS, el)}


def bench_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    u0 = workload(0)
    from oracle import oracle as O
    cfg = O.Cfg1D.make(O.EULER, NX, 0.0, 1.0, O.BC_OUTFLOW)
    sample_steps = 10
    u = u0.copy()
    for _ in range(args.warmup):
        O.run1d(cfg, u, nsteps=sample_steps, cfl=CFL)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u, _, _ = O.run1d(cfg, u, nsteps=sample_steps, cfl=CFL)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = NX * 3 * sample_steps * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "1D Euler two-state, 65536 cells, outflow, CFL %.1f; each step "
                               "%d of the %d RK steps (bounded sample)" % (CFL, sample_steps, RK_STEPS),
                   "seed": SEED},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d RK steps x %d timed steps on 65536 cells, 1 thread"
                                   % (sample_steps, args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def bench_hweno(args):
    import torch
    import torch.distributed as dist

    from paper_2002_08816_gb300 import hweno as H
    import __graft_entry__

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    u0 = workload(rank)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()

    results = {}
    for prec_name, prec in (("fp32", H.HWENO_FP32), ("fp64", H.HWENO_FP64)):
        cfg = H.make_config(1, H.HWENO_EULER, NX, x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW, cfl=CFL,
                            precision=prec)
        h = H.hweno_create(cfg, s)
        dt = torch.float32 if prec == H.HWENO_FP32 else torch.float64
        dev_in = torch.from_numpy(u0).to("cuda", dt).contiguous()
        host_in = torch.from_numpy(u0).to(dt).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()

        def one_step():
            H.hweno_set_state(h, dev_in.data_ptr(), prec, True)
            H.hweno_step(h, RK_STEPS, -1.0, wait=False)

        # the library's autotuner picks threads per CTA and graph or persistent
        # launches for this workload (untimed)
        H.hweno_set_state(h, dev_in.data_ptr(), prec, True)
        choice = H.hweno_autotune(h, 100)
        for _ in range(args.warmup):
            one_step()
        torch.cuda.synchronize()
        t_end = H.hweno_step(h, 0, -1.0)  # status check of the warm-up runs
        assert t_end > 0.0
        st_w = H.hweno_stats(h)
        assert st_w["steps"] == RK_STEPS

        # device-resident timing: L2 flushed between timed steps, events on the stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sampler = ClockSampler(local) if prec_name == "fp32" else None
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.__enter__()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            one_step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = [a.elapsed_time(b) for a, b in ev]
        H.hweno_step(h, 0, -1.0)  # raises on a non-physical run
        stats = H.hweno_stats(h)
        tot_s = max_over_ranks(sum(ms) / 1e3)

        # end to end through the public API with host buffers (pinned)
        e2e_ms = []
        for k in range(max(1, min(args.steps, 3))):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            H.hweno_set_state(h, host_in.data_ptr(), prec, False)
            H.hweno_step(h, RK_STEPS, -1.0, wait=False)
            H.hweno_get_state(h, host_out.data_ptr(), prec, False)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e_s = max_over_ranks(sum(e2e_ms) / 1e3)
        final = np.empty(u0.shape, dtype=np.float64)  # the state after RK_STEPS steps
        H.hweno_get_state(h, final.ctypes.data, H.HWENO_FP64, False)
        H.hweno_destroy(h)
        cells = NX * 3 * RK_STEPS
        results[prec_name] = {
            "value": job_value(ws, cells * args.steps, tot_s),
            "ms_per_step": 1e3 * tot_s / args.steps,
            "stage_us": 1e6 * tot_s / (args.steps * 3 * RK_STEPS),
            "e2e": job_value(ws, cells * len(e2e_ms), e2e_s),
            "troubled_frac": stats["troubled"] / float(3 * RK_STEPS * NX),
            "bytes_h2d": host_in.numel() * host_in.element_size(),
            "clocks": sampler.summary() if sampler else None,
            "execution": {"threads_per_cta": choice[0], "cells_per_tile": choice[0] - 6,
                          "launch": "persistent" if choice[1] else "per-stage graphs",
                          "chosen_by": "hweno_autotune"},
            "final": final,
        }

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(u0)
    if rank != 0:
        dist.destroy_process_group() if ws > 1 else None
        return
    r = results["fp32"]
    peak, peak_kind = peaks()
    # per-field error of the FP32 path against the FP64 path after the 2000
    # steps (the FP64 path matches the FP64 oracle to 1e-12 in the parity tests)
    a32, a64 = results["fp32"].pop("final"), results["fp64"].pop("final")
    field_err = {}
    for c, name in enumerate(("rho", "m", "E")):
        for m, mom in enumerate(("average", "first_moment")):
            d = np.abs(a32[c, m] - a64[c, m])
            field_err["%s_%s" % (name, mom)] = {
                "L1": float(d.mean()), "Linf": float(d.max()),
                "rel_L1": float(d.sum() / max(np.abs(a64[c, m]).sum(), 1e-300))}
    persistent = r["execution"]["launch"] == "persistent"
    per_launch = BYTES_PER_CELL_STAGE["fp32"] * NX
    achieved = per_launch / (r["stage_us"] * 1e-6) / 1e9
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "1D Euler two-state, 65536 cells, outflow, 2000 SSP-RK3 steps, "
                               "CFL 0.5, FP32 (time accumulated in FP64)",
                   "seed": SEED, "l2": "flushed (512 MiB write) between timed steps",
                   "parallelism": "one independent instance per GPU"},
        "fp64": {"value": results["fp64"]["value"], "ms_per_step": results["fp64"]["ms_per_step"],
                 "e2e": results["fp64"]["e2e"], "execution": results["fp64"]["execution"],
                 "bound": "FP64 pipe (~80 % active under ncu)"},
        "troubled_frac": r["troubled_frac"],
        "fp32_vs_fp64": field_err,
        "execution": r["execution"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": TRAFFIC_1D_FP32.get((r["execution"]["threads_per_cta"],
                                                     r["execution"]["launch"])),
                     "kernel": "%s<float,3,%d threads>" % (
                         "run1d_kernel" if persistent else "stage1d_kernel",
                         r["execution"]["threads_per_cta"]),
                     "note": ("avg stage time = timed region / 6000 stages (one persistent launch "
                              "per step, traffic per stage) " if persistent else
                              "avg stage-launch time = timed region / 6000 launches ")
                             + "; peak %s" % peak_kind},
        "cpu_baseline": cpu,
        "e2e": {"value": r["e2e"], "unit": UNIT, "h2d_bytes_per_step": r["bytes_h2d"],
                "d2h_bytes_per_step": r["bytes_h2d"]},
        # per step: alpha, convert and two scalar resets, plus the stage
        # launches or the one persistent launch
        "gpu_launches": args.steps * ((1 if persistent else 3 * RK_STEPS) + 4),
        "clocks": r["clocks"],
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- 2D workload

NX2 = 4096
RK_STEPS_2D = 100
SEED_2D = 2026
CFL_2D = 0.5
COEF_HDR = os.path.join(ROOT, "paper_2002_08816_gb300", "csrc", "hweno2d_coef.cuh")


def flops_per_cell_stage_2d(ng, ncomp=4):
    """FP32 operations of one smooth 2D cell-stage, counted on the operations
    the method needs (halo recomputation excluded): the linear p0 maps of the
    generated code (one FMA = 2 flops per nonzero coefficient) for the 4 ng
    interface and ng^2 interior points of every component, the Lax-Friedrichs
    flux of each of the cell's own 2 ng interface points (Euler: two fluxes of
    15 flops and 16 for the combination; Burgers: two u^2/2 and 4), f and g at
    the interior points (Euler 2 x 15 + 16; Burgers 2 + 4), the right-hand-side
    sums (6 per quadrature point and component plus 10) and the Runge-Kutta
    combination (4 per moment)."""
    import re
    txt = open(COEF_HDR).read()
    nnz = 0
    for name in ("p0_faces_ng%d" % ng, "p0_interior_ng%d" % ng):
        body = re.search(r"void %s\(const R\* d, R\* o\) \{(.*?)\n\}" % name, txt, re.S).group(1)
        nnz += len(re.findall(r"\* d\[", body))
    pt = 46 if ncomp == 4 else 8
    return (2 * ncomp * nnz + 2 * ng * pt + ng * ng * pt + ncomp * (6 * 3 * ng + 10)
            + 4 * 3 * ncomp)


def bench_euler2d(args):
    """2D Euler, 4096 x 4096 periodic [0, 10]^2, isentropic vortex plus seeded
    density modes, FP32, RK_STEPS_2D steps per bench step (state > L2)."""
    import torch
    import torch.distributed as dist

    from paper_2002_08816_gb300 import hweno as H
    from paper_2002_08816_gb300 import workloads as W
    import __graft_entry__

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    ng = args.n_gauss or 2
    burgers = args.workload == "burgers2d"
    ncomp = 1 if burgers else 4
    if burgers:  # Example 3.9's data (0.5 + sin(pi (x + y)/2) on [0, 4]^2), past the shock
        u0 = W.burgers_sine_2d(NX2, NX2, npts=2).astype(np.float32)
        cfg = H.make_config(2, H.HWENO_BURGERS, NX2, NX2, x0=0.0, x1=4.0, y0=0.0, y1=4.0,
                            bc=H.HWENO_BC_PERIODIC, cfl=0.6, precision=H.HWENO_FP32, n_gauss=ng)
    else:
        u0 = W.euler_vortex_modes_2d(NX2, NX2, seed=SEED_2D + rank, npts=2).astype(np.float32)
        cfg = H.make_config(2, H.HWENO_EULER, NX2, NX2, x0=0.0, x1=10.0, y0=0.0, y1=10.0,
                            bc=H.HWENO_BC_PERIODIC, cfl=CFL_2D, precision=H.HWENO_FP32, n_gauss=ng)
    h = H.hweno_create(cfg, stream.cuda_stream)
    dev = torch.from_numpy(u0).to("cuda")
    host_in = torch.from_numpy(u0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def one_step():
        H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
        H.hweno_step(h, RK_STEPS_2D, -1.0, wait=False)

    for _ in range(args.warmup):
        one_step()
    H.hweno_step(h, 0, -1.0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.__enter__()
    for k in range(args.steps):
        ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sampler.__exit__(None, None, None)
    ms = [a.elapsed_time(b) for a, b in ev]
    H.hweno_step(h, 0, -1.0)
    st = H.hweno_stats(h)
    tot = max_over_ranks(sum(ms) / 1e3)
    # end to end from pinned host buffers
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    H.hweno_set_state(h, host_in.data_ptr(), H.HWENO_FP32, False)
    H.hweno_step(h, RK_STEPS_2D, -1.0, wait=False)
    H.hweno_get_state(h, host_out.data_ptr(), H.HWENO_FP32, False)
    b.record(stream)
    b.synchronize()
    e2e_s = a.elapsed_time(b) / 1e3
    H.hweno_destroy(h)
    quad = None
    if not burgers:
        # the second run of the workload: four constant quadrants drawn from
        # the seed (shocks and troubled cells), one timed bench step
        uq = W.euler_quadrants_2d(NX2, NX2, seed=SEED_2D + rank, npts=2).astype(np.float32)
        devq = torch.from_numpy(uq).to("cuda")
        del uq
        hq = H.hweno_create(cfg, stream.cuda_stream)
        try:
            H.hweno_set_state(hq, devq.data_ptr(), H.HWENO_FP32, True)
            H.hweno_step(hq, RK_STEPS_2D, -1.0)  # warm-up (builds the graphs)
            H.hweno_set_state(hq, devq.data_ptr(), H.HWENO_FP32, True)
            qa, qb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            qa.record(stream)
            H.hweno_step(hq, RK_STEPS_2D, -1.0, wait=False)
            qb.record(stream)
            qb.synchronize()
            H.hweno_step(hq, 0, -1.0)
            q_s = max_over_ranks(qa.elapsed_time(qb) / 1e3)
            ncs = NX2 * NX2 * 3 * RK_STEPS_2D
            quad = {"value": job_value(ws, ncs, q_s), "ms_per_step": 1e3 * q_s,
                    # set_state resets the counters: these are the timed step's
                    "troubled_frac": H.hweno_stats(hq)["troubled"] / float(ncs),
                    "data": "four constant quadrants (rho, u, v, p) drawn from the seed, same grid, "
                            "steps and CFL; one timed bench step after one warm-up step"}
        finally:
            H.hweno_destroy(hq)
        del devq
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    cells = NX2 * NX2 * 3 * RK_STEPS_2D
    stage_s = tot / (args.steps * 3 * RK_STEPS_2D)
    clocks = sampler.summary()
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the sampled SM clock
    flops = flops_per_cell_stage_2d(ng, ncomp) * NX2 * NX2
    byts = (8 * 3 * 4 * ncomp / 3) * NX2 * NX2  # 8S/3, S = 3 moments x ncomp x 4 B
    hbm, peak_kind = peaks()
    t_alu = flops / (fp32_peak * 1e12)
    t_hbm = byts / (hbm * 1e9)
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": flops / stage_s / 1e12, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": t_alu / stage_s,
                "traffic": TRAFFIC_2D_NG2 if (ng == 2 and not burgers) else None,
                "note": "FP32 peak = 152 SMs x 128 lanes x 2 flops x sampled SM clock; "
                        "%d flops per smooth cell-stage" % flops_per_cell_stage_2d(ng, ncomp)}
    else:
        roof = {"bound": "hbm", "achieved": byts / stage_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": t_hbm / stage_s,
                "traffic": TRAFFIC_2D_NG2 if (ng == 2 and not burgers) else None,
                "note": "peak %s" % peak_kind}
    roof["kernel"] = "stage2d_kernel<float,%d,%d>" % (ncomp, ng)
    line = {
        "metric": METRIC, "value": job_value(ws, cells * args.steps, tot), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": ("2D Burgers 4096x4096 periodic on [0,4]^2, 0.5 + sin(pi (x+y)/2) "
                                "(Example 3.3/3.9 data), %d RK3 steps, %d Gauss points, CFL 0.6, "
                                "FP32" % (RK_STEPS_2D, ng)) if burgers else
                               ("2D Euler 4096x4096 periodic, vortex + 8 density modes, %d RK3 "
                                "steps, %d Gauss points, CFL %.1f, FP32" % (RK_STEPS_2D, ng, CFL_2D)),
                   "seed": SEED_2D, "l2": "state (%d MB) larger than L2" % (u0.nbytes // 10 ** 6)},
        "stage_ms": stage_s * 1e3,
        # set_state resets the counters: the last bench step's troubled cell-stages
        "troubled_frac": st["troubled"] / float(cells),
        "quadrants": quad,
        "roofline": roof,
        "e2e": {"value": cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": host_in.numel() * 4,
                "d2h_bytes_per_step": host_in.numel() * 4},
        "gpu_launches": args.steps * (3 * RK_STEPS_2D + 4),
        "clocks": clocks,
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- adjoint workload

NX_ADJ = 1024
STEPS_ADJ = 200
EVERY_ADJ = 20
SEED_ADJ = 4242


def bench_adjoint2d(args):
    """Gradient of sum(rho^2) after STEPS_ADJ steps with respect to the initial
    moments: 2D Euler 1024 x 1024 periodic [0, 10]^2, vortex plus density
    modes, FP32, forward with the tape (checkpoint every EVERY_ADJ steps), then
    the checkpointed adjoint.  Reports forward, backward and their ratio."""
    import torch

    from paper_2002_08816_gb300 import hweno as H
    from paper_2002_08816_gb300 import workloads as W
    import __graft_entry__

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    ng = args.n_gauss or 3
    n = NX_ADJ
    u0 = W.euler_vortex_modes_2d(n, n, seed=SEED_ADJ + rank).astype(np.float32)
    cfg = H.make_config(2, H.HWENO_EULER, n, n, x0=0.0, x1=10.0, y0=0.0, y1=10.0,
                        bc=H.HWENO_BC_PERIODIC, cfl=CFL_2D, precision=H.HWENO_FP32, n_gauss=ng)
    h = H.hweno_create(cfg, stream.cuda_stream)
    dev = torch.from_numpy(u0).to("cuda")
    uN = torch.empty_like(dev)
    grad = torch.empty_like(dev)
    seed_grad = torch.zeros_like(dev)

    def forward():
        H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
        H.hweno_record(h, STEPS_ADJ, EVERY_ADJ)
        H.hweno_get_state(h, uN.data_ptr(), H.HWENO_FP32, True)

    def backward():
        seed_grad[0, 0] = 2.0 * uN[0, 0]  # d sum(rho^2) / d u_N
        H.hweno_backward(h, seed_grad.data_ptr(), grad.data_ptr(), H.HWENO_FP32, True)

    for _ in range(args.warmup):
        forward()
        backward()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.__enter__()
    tf, tb = [], []
    for _ in range(args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        forward()
        e[1].record(stream)
        backward()
        e[2].record(stream)
        e[2].synchronize()
        tf.append(e[0].elapsed_time(e[1]) / 1e3)
        tb.append(e[1].elapsed_time(e[2]) / 1e3)
    # one adjoint stage (kernels A and B) on the final state, and one forward
    # stage, timed alone
    flags = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
    lam = torch.randn_like(dev)
    out = torch.empty_like(dev)
    reps = 20
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    H.hweno_rhs(h, uN.data_ptr(), out.data_ptr(), flags.data_ptr(), 0)
    a.record(stream)
    for _ in range(reps):
        H.hweno_rhs_vjp(h, uN.data_ptr(), flags.data_ptr(), 1.0, 1.0, lam.data_ptr(), out.data_ptr())
    b.record(stream)
    b.synchronize()
    adj_stage_s = a.elapsed_time(b) / 1e3 / reps
    sampler.__exit__(None, None, None)
    H.hweno_destroy(h)
    if rank != 0:
        return
    t_f, t_b = statistics.median(tf), statistics.median(tb)
    cells = n * n * 3 * STEPS_ADJ
    clocks = sampler.summary()
    line = {
        "metric": "cell-stages/s of forward + adjoint (gradient of sum rho^2)", "value": cells / (t_f + t_b),
        "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * (t_f + t_b), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "adjoint: 2D Euler 1024x1024 periodic, vortex + 8 density modes, "
                               "loss sum(rho^2) after %d RK3 steps, checkpoint every %d, "
                               "%d Gauss points, FP32" % (STEPS_ADJ, EVERY_ADJ, ng),
                   "seed": SEED_ADJ, "l2": "state 50 MB, tape and segment states > L2"},
        "forward_ms": t_f * 1e3, "backward_ms": t_b * 1e3,
        "adjoint_over_forward": t_b / t_f,
        "adjoint_stage_ms": adj_stage_s * 1e3,
        "forward_cell_stages_per_s": cells / t_f,
        "clocks": clocks,
        # forward and recomputed stages, two adjoint kernels per stage, one
        # wave-speed launch per segment, and the state conversions and resets
        "gpu_launches": args.steps * (3 * STEPS_ADJ * 2 + 6 * STEPS_ADJ + STEPS_ADJ // EVERY_ADJ + 6),
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------- batched 1D workload

N_BATCH = 512
RK_STEPS_BATCH = 500
SEED_BATCH = 77


def bench_batch1d(args):
    """512 independent 1D Euler instances, cell counts log-uniform in
    [256, 16384], two-state data, FP32, RK_STEPS_BATCH steps each, advanced in
    shared launches; compared with one handle per instance on an evenly spread
    subset of 32 instances (the per-instance time is launch-bound, so it is
    scaled to 512 instances by their count)."""
    import torch

    from paper_2002_08816_gb300 import hweno as H
    from paper_2002_08816_gb300 import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    sizes = [int(v) for v in W.batch_sizes_1d(N_BATCH, seed=SEED_BATCH)]
    states = [W.euler_two_state_1d(n, seed=SEED_BATCH + b).astype(np.float32)
              for b, n in enumerate(sizes)]
    cells = sum(sizes)
    cfg = H.make_config(1, H.HWENO_EULER, 4, x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW, cfl=CFL,
                        precision=H.HWENO_FP32)
    h = H.hweno_create_batch(cfg, sizes, stream.cuda_stream)
    dev = torch.from_numpy(np.concatenate([s.reshape(-1) for s in states])).to("cuda")

    def one_step():
        H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
        H.hweno_step(h, RK_STEPS_BATCH, -1.0, wait=False)

    H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
    choice = H.hweno_autotune(h, 20)  # tile size and launch kind, untimed
    for _ in range(args.warmup):
        one_step()
    H.hweno_step(h, 0, -1.0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(0)
    sampler.__enter__()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sampler.__exit__(None, None, None)
    H.hweno_step(h, 0, -1.0)
    H.hweno_destroy(h)
    tot = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    # one handle per instance, on 32 instances spread over the size range
    order = np.argsort(sizes)
    pick = [int(order[k]) for k in np.linspace(0, N_BATCH - 1, 32).round().astype(int)]
    handles = []
    for b in pick:
        c1 = H.make_config(1, H.HWENO_EULER, sizes[b], x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW,
                           cfl=CFL, precision=H.HWENO_FP32)
        hb = H.hweno_create(c1, stream.cuda_stream)
        d = torch.from_numpy(states[b]).to("cuda")
        handles.append((hb, d))
    for hb, d in handles:  # warm-up (graph capture)
        H.hweno_set_state(hb, d.data_ptr(), H.HWENO_FP32, True)
        H.hweno_step(hb, 40, -1.0, wait=False)
    torch.cuda.synchronize()
    a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for hb, d in handles:
        H.hweno_set_state(hb, d.data_ptr(), H.HWENO_FP32, True)
        H.hweno_step(hb, RK_STEPS_BATCH, -1.0, wait=False)
    b2.record(stream)
    b2.synchronize()
    sub_s = a.elapsed_time(b2) / 1e3
    for hb, _ in handles:
        H.hweno_destroy(hb)
    per_inst_s = sub_s * N_BATCH / len(pick)
    value = cells * 3 * RK_STEPS_BATCH * args.steps / tot
    hbm, peak_kind = peaks()
    stage_s = tot / (args.steps * 3 * RK_STEPS_BATCH)
    achieved = BYTES_PER_CELL_STAGE["fp32"] * cells / stage_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched 1D Euler: 512 instances, cells log-uniform in "
                               "[256, 16384] (%d cells), two-state data, %d RK3 steps each, "
                               "CFL %.1f, FP32, all instances in shared launches"
                               % (cells, RK_STEPS_BATCH, CFL),
                   "seed": SEED_BATCH, "l2": "flushed (512 MiB write) between timed steps"},
        "per_instance": {"ms_per_step_estimate": 1e3 * per_inst_s,
                         "value_estimate": cells * 3 * RK_STEPS_BATCH / per_inst_s,
                         "how": "one handle per instance (CUDA graphs of 32 steps), 32 instances "
                                "spread over the sizes, %.1f ms, scaled by 512/32" % (1e3 * sub_s)},
        "speedup_vs_per_instance": per_inst_s / (tot / args.steps),
        "execution": {"threads_per_cta": choice[0], "cells_per_tile": choice[0] - 6,
                      "launch": "persistent" if choice[1] else "per-stage graphs",
                      "chosen_by": "hweno_autotune"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": TRAFFIC_BATCH_FP32.get((choice[0], bool(choice[1]))),
                     "kernel": "%s<float,3,batch,%d threads>" % (
                         "run1d_kernel" if choice[1] else "stage1d_kernel", choice[0]),
                     "note": "avg stage time = timed region (set_state included) / %d stages; "
                             "the %d MB state fits in L2; peak %s"
                             % (3 * RK_STEPS_BATCH, cells * 24 // 10 ** 6, peak_kind)},
        "gpu_launches": args.steps * (3 * RK_STEPS_BATCH + 5),
        "clocks": sampler.summary(),
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hweno", choices=["hweno", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="euler1d",
                    choices=["euler1d", "euler2d", "burgers2d", "batch1d", "adjoint2d"],
                    help="euler1d: the headline 65536-cell 1D workload; euler2d: the "
                         "4096 x 4096 2D Euler workload; burgers2d: 2D Burgers (Example "
                         "3.9's data) at 4096 x 4096; batch1d: 512 uneven 1D instances; "
                         "adjoint2d: gradient through 200 steps of 2D Euler at 1024 x 1024")
    ap.add_argument("--n-gauss", type=int, default=None, choices=[2, 3],
                    help="Gauss points per direction (2D): default 2 for euler2d (its "
                         "configuration), 3 for adjoint2d (the paper's)")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload in ("euler2d", "burgers2d"):
        bench_euler2d(args)
    elif args.workload == "batch1d":
        bench_batch1d(args)
    elif args.workload == "adjoint2d":
        bench_adjoint2d(args)
    else:
        bench_hweno(args)


if __name__ == "__main__":
    main()
