"""Benchmark of the hybrid HWENO time stepper on GB300.

Headline workload (one bench step): the seeded two-state 1D Euler problem,
gamma 1.4, 65536 cells on [0, 1] with outflow ends, advanced 2000 third-order
TVD Runge-Kutta steps (6000 stages, 3.93e8 cell-stages) at CFL 0.5, FP32 bulk
arithmetic (the global CFL reduction, dt and the time in FP64).  The metric is
cell-updates per second counted per Runge-Kutta stage.  The FP64 path is timed
on the same workload and reported beside it.  At one GPU the default run also
measures, each in its own sub-record of the same JSON line ("workloads"), the
other workloads: 2D Euler 4096 x 4096 with 2 and 3 Gauss points and its
four-quadrant second run, 512 uneven batched 1D instances against 512
per-instance handles, the 2D adjoint at 1024 x 1024, and a 1D workload with a
paper-like share of troubled cells; and the measured FP32 / FP64 FMA peaks of
the GPU ("alu_peaks").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hweno|reference]
                  [--workload euler1d|euler2d|burgers2d|batch1d|adjoint2d|troubled1d]
                  [--headline-only] [--no-cpu-baseline]

--impl reference times the FP64 C oracle on the host cores (all of them, its
OpenMP build) on a bounded sample of the same workload.  Under torchrun each
rank advances its own seeded instance (no data-path collective): weak scaling.
"""

import argparse
import copy
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
BYTES_PER_CELL_STAGE = {"fp32": 8 * 24 / 3, "fp64": 8 * 48 / 3, "fp32c": 8 * 36 / 3}
# DRAM bytes (read + write) per stage from ncu captures of the current kernels,
# summarised under profiles/ (None where no capture of the current build exists):
# the resident launch reads the state once per launch: a 2000-step (6000-stage)
# capture over its stages; FP32C also reads the averages' low parts
TRAFFIC_1D_FP32 = {(256, "resident"): (2069504 + 63488) / 6000}
TRAFFIC_1D_FP32C = {(256, "resident"): (2937856 + 55808) / 6000}
# the troubled-share workload's resident launch: a 200-step (600-stage) capture
TRAFFIC_TROUBLED_1D = {(256, "resident"): (1767936 + 53248) / 600}
# the batched workload, 128-thread per-stage launches: the mean of the three
# stages of one step, cold L2
TRAFFIC_BATCH_FP32 = {(128, "per-stage graphs"): (48942336 + 43494656 + 96712960 + 22568192
                                                  + 96711424 + 21799936) / 3}
# 2D, 2 Gauss points: a 2048^2 capture (the three stages of one step) scaled
# by the cell count to 4096^2 (the bytes per cell do not depend on the grid)
TRAFFIC_2D_NG2 = 4 * (202326016 + 350454528 + 403358976 + 173675008 + 403536384
                      + 175169536) / 3
L2_FLUSH_BYTES = 512 << 20
# hweno_autotune's launch kinds and the kernel each one times
LAUNCH_KIND = {0: "per-stage graphs", 1: "persistent", 2: "resident"}
KERNEL_OF_LAUNCH = {"per-stage graphs": "stage1d_kernel", "persistent": "run1d_kernel",
                    "resident": "resident1d_kernel"}


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


def field_errors(a, ref, names=("rho", "m", "E"), moments=("average", "first_moment")):
    """Per field (component x moment) L1, L-infinity and relative L1 of a
    against ref, both [C][M][cells]; and the first moments' L1 relative to the
    L1 of the averages / 4 (|vbar| <= max |u| / 4: their natural scale)."""
    out = {}
    for c, name in enumerate(names):
        for m, mom in enumerate(moments):
            d = np.abs(a[c, m] - ref[c, m])
            e = {"L1": float(d.mean()), "Linf": float(d.max()),
                 "rel_L1": float(d.sum() / max(np.abs(ref[c, m]).sum(), 1e-300))}
            if m > 0:
                e["L1_over_avg_scale"] = float(d.sum() / max(np.abs(ref[c, 0]).sum() / 4, 1e-300))
            out["%s_%s" % (name, mom)] = e
    return out


# ----------------------------------------------------------------------------- CPU baseline

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


def run_oracle_full(u_in):
    """The oracle's OpenMP build on all host cores over the whole workload
    (2000 RK steps of the 65536-cell state, FP64): the all-core CPU baseline,
    and the FP64 reference state the GPU runs are measured against."""
    from oracle import oracle as O
    cores = O.threads(os.cpu_count() or 1)
    cfg = O.Cfg1D.make(O.EULER, NX, 0.0, 1.0, O.BC_OUTFLOW)
    t0 = time.perf_counter()
    u, t, nt = O.run1d(cfg, u_in, nsteps=RK_STEPS, cfl=CFL, omp=True)
    el = time.perf_counter() - t0
    return u, t, nt, {"value": NX * 3 * RK_STEPS / el, "unit": UNIT, "cores": cores,
                      "kind": "oracle",
                      "sample": "the whole workload (%d RK steps of 65536 cells), FP64, OpenMP "
                                "build on %d threads, %.1f s" % (RK_STEPS, cores, el)}


def bench_reference(args):
    """The oracle as it stands on the host cores (its OpenMP build on all of
    them) on bounded samples of the headline workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    u0 = workload(0)
    from oracle import oracle as O
    cores = O.threads(os.cpu_count() or 1)
    cfg = O.Cfg1D.make(O.EULER, NX, 0.0, 1.0, O.BC_OUTFLOW)
    sample_steps = 40
    u = u0.copy()
    for _ in range(args.warmup):
        O.run1d(cfg, u, nsteps=sample_steps, cfl=CFL, omp=True)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u, _, _ = O.run1d(cfg, u, nsteps=sample_steps, cfl=CFL, omp=True)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = NX * 3 * sample_steps * args.steps / tot
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "1D Euler two-state, 65536 cells, outflow, CFL %.1f; each step "
                               "%d of the %d RK steps (bounded sample)" % (CFL, sample_steps, RK_STEPS),
                   "seed": SEED},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d RK steps x %d timed steps on 65536 cells, OpenMP build, "
                                   "%d threads" % (sample_steps, args.steps, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ----------------------------------------------------------------------------- ALU peaks

def alu_peaks():
    """FP32 and FP64 FMA throughput of this GPU, measured by the library's
    microbenchmark (hweno_fma_peak) with the SM clock sampled meanwhile."""
    import torch
    from paper_2002_08816_gb300 import hweno as H
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.__enter__()
    f32 = max(H.hweno_fma_peak(0, 20000) for _ in range(3))
    f64 = max(H.hweno_fma_peak(1, 300) for _ in range(2))
    f32x2 = max(H.hweno_fma_peak(2, 10000) for _ in range(3))
    sampler.__exit__(None, None, None)
    return {"fp32_tflops": f32 / 1e12, "fp64_tflops": f64 / 1e12,
            "fp32_packed_tflops": f32x2 / 1e12,
            "sm_count": props.multi_processor_count, "clocks": sampler.summary(),
            "how": "hweno_fma_peak: 8 independent FMA chains per thread (packed: 8 chains of "
                   "fma.rn.f32x2 pairs), a grid filling every SM, CUDA events, best of 3 (FP32) "
                   "/ 2 (FP64); the FP32 roofline divides by the larger of the two FP32 figures"}


# ----------------------------------------------------------------------------- headline (1D)

def run_1d(H, s, stream, u0, prec, steps, warmup, flush, sampler=None, autotune=True):
    """One precision of the headline workload: autotuned execution, device-
    resident timing (L2 flushed between timed steps), end to end from pinned
    host buffers; returns the timings and the final state."""
    import torch
    cfg = H.make_config(1, H.HWENO_EULER, NX, x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW, cfl=CFL,
                        precision=prec)
    h = H.hweno_create(cfg, s)
    # the state's element type: FP32 for both FP32 precisions (HWENO_FP32C then
    # starts from zero low parts: the same input the FP32 path and the oracle see)
    sdt = H.HWENO_FP64 if prec == H.HWENO_FP64 else H.HWENO_FP32
    dt = torch.float64 if sdt == H.HWENO_FP64 else torch.float32
    dev_in = torch.from_numpy(u0).to("cuda", dt).contiguous()
    host_in = torch.from_numpy(u0).to(dt).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def one_step():
        H.hweno_set_state(h, dev_in.data_ptr(), sdt, True)
        H.hweno_step(h, RK_STEPS, -1.0, wait=False)

    # the library's autotuner picks threads per CTA and the launch kind for
    # this workload (untimed)
    H.hweno_set_state(h, dev_in.data_ptr(), sdt, True)
    choice = H.hweno_autotune(h, 100) if autotune else (256, 0)
    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    assert H.hweno_step(h, 0, -1.0) > 0.0  # status check of the warm-up runs
    assert H.hweno_stats(h)["steps"] == RK_STEPS
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    if sampler:
        sampler.__enter__()
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__(None, None, None)
    ms = [a.elapsed_time(b) for a, b in ev]
    H.hweno_step(h, 0, -1.0)  # raises on a non-physical run
    stats = H.hweno_stats(h)
    e2e_ms = []
    for k in range(max(1, min(steps, 3))):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        H.hweno_set_state(h, host_in.data_ptr(), sdt, False)
        H.hweno_step(h, RK_STEPS, -1.0, wait=False)
        H.hweno_get_state(h, host_out.data_ptr(), sdt, False)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    final = np.empty(u0.shape, dtype=np.float64)
    H.hweno_get_state(h, final.ctypes.data, H.HWENO_FP64, False)
    H.hweno_destroy(h)
    return {"ms": ms, "e2e_ms": e2e_ms, "stats": stats, "choice": choice, "final": final,
            "bytes_h2d": host_in.numel() * host_in.element_size()}


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
    u0r = u0.astype(np.float32).astype(np.float64)  # the input both the FP32 path and the oracle see
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()

    cells = NX * 3 * RK_STEPS
    res = {}
    for name, prec in (("fp32", H.HWENO_FP32), ("fp32c", H.HWENO_FP32C), ("fp64", H.HWENO_FP64)):
        barrier()
        sampler = ClockSampler(local) if name == "fp32" else None
        r = run_1d(H, s, stream, u0 if name == "fp64" else u0r, prec, args.steps, args.warmup,
                   flush, sampler)
        tot_s = max_over_ranks(sum(r["ms"]) / 1e3)
        e2e_s = max_over_ranks(sum(r["e2e_ms"]) / 1e3)
        r.update({"value": job_value(ws, cells * args.steps, tot_s),
                  "ms_per_step": 1e3 * tot_s / args.steps,
                  "stage_us": 1e6 * tot_s / (args.steps * 3 * RK_STEPS),
                  "e2e": job_value(ws, cells * len(r["e2e_ms"]), e2e_s),
                  "clocks": sampler.summary() if sampler else None,
                  "execution": {"threads_per_cta": r["choice"][0],
                                "launch": LAUNCH_KIND[r["choice"][1]],
                                "chosen_by": "hweno_autotune"}})
        res[name] = r
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None
    r = res["fp32"]
    launch = r["execution"]["launch"]
    peak, peak_kind = peaks()
    per_launch = BYTES_PER_CELL_STAGE["fp32"] * NX
    achieved = per_launch / (r["stage_us"] * 1e-6) / 1e9
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "1D Euler two-state, 65536 cells, outflow, 2000 SSP-RK3 steps, "
                               "CFL 0.5, FP32 (CFL reduction, dt and time in FP64)",
                   "seed": SEED, "l2": "flushed (512 MiB write) between timed steps",
                   "parallelism": "one independent instance per GPU"},
        "stage_us": r["stage_us"],
        "fp64": {"value": res["fp64"]["value"], "ms_per_step": res["fp64"]["ms_per_step"],
                 "stage_us": res["fp64"]["stage_us"], "e2e": res["fp64"]["e2e"],
                 "execution": res["fp64"]["execution"]},
        # FP32 arithmetic with float-pair averages (HWENO_FP32C), same input
        "fp32c": {"value": res["fp32c"]["value"], "ms_per_step": res["fp32c"]["ms_per_step"],
                  "stage_us": res["fp32c"]["stage_us"], "e2e": res["fp32c"]["e2e"],
                  "execution": res["fp32c"]["execution"],
                  "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak,
                               "achieved": BYTES_PER_CELL_STAGE["fp32c"] * NX
                               / (res["fp32c"]["stage_us"] * 1e-6) / 1e9,
                               "frac": BYTES_PER_CELL_STAGE["fp32c"] * NX
                               / (res["fp32c"]["stage_us"] * 1e-6) / 1e9 / peak,
                               "traffic": TRAFFIC_1D_FP32C.get(
                                   (res["fp32c"]["execution"]["threads_per_cta"],
                                    res["fp32c"]["execution"]["launch"])),
                               "note": "algorithmic 96 B per cell-stage (the averages as float "
                                       "pairs: 36 B per cell) x 65536 cells per stage"}},
        "troubled_frac": r["stats"]["troubled"] / float(cells),
        "execution": r["execution"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": TRAFFIC_1D_FP32.get((r["execution"]["threads_per_cta"], launch)),
                     "kernel": "%s<float,3,%d threads>" % (KERNEL_OF_LAUNCH[launch],
                                                           r["execution"]["threads_per_cta"]),
                     "note": "algorithmic 64 B per cell-stage x 65536 cells per stage over the "
                             "average stage time (timed region / 6000 stages); peak %s" % peak_kind},
        "e2e": {"value": r["e2e"], "unit": UNIT, "h2d_bytes_per_step": r["bytes_h2d"],
                "d2h_bytes_per_step": r["bytes_h2d"]},
        # per step: the set_state conversion and scalar reset, its wave-speed
        # kernel and hweno_step's scalar reset, plus the stage launches or the
        # one persistent / resident launch
        "gpu_launches": args.steps * ((3 * RK_STEPS if launch == "per-stage graphs" else 1) + 4),
        "clocks": r["clocks"],
    }
    if not args.no_cpu_baseline:
        # the oracle as it stands: a bounded single-thread sample, and the whole
        # workload on all host cores (OpenMP build), whose final state is the FP64
        # reference of the accuracy figures
        single = run_cpu_baseline(u0r)
        ref, t_ref, nt_ref, allc = run_oracle_full(u0r)
        line["cpu_baseline"] = dict(single, all_cores=allc)
        line["fp32_vs_oracle"] = field_errors(res["fp32"]["final"], ref)
        line["fp32_vs_oracle"]["note"] = (
            "after the 2000 shocked steps, same FP32-rounded input; rel_L1 per field and the "
            "first moments' L1 over the averages' L1 / 4")
        line["fp32c_vs_oracle"] = field_errors(res["fp32c"]["final"], ref)
        line["fp32c_vs_oracle"]["note"] = "HWENO_FP32C, same input and reference as fp32_vs_oracle"
        # conditioning: the FP64 GPU path from the unrounded input against the
        # oracle from the FP32-rounded one (one rounding of the input, no FP32
        # arithmetic)
        line["fp64_unrounded_vs_oracle"] = field_errors(res["fp64"]["final"], ref)
        line["time_vs_oracle"] = {"fp32": abs(r["stats"]["t"] - t_ref) / t_ref,
                                  "fp32c": abs(res["fp32c"]["stats"]["t"] - t_ref) / t_ref}
    if ws > 1:
        dist.destroy_process_group()
    return line


# ----------------------------------------------------------------------------- 2D workload

NX2 = 4096
RK_STEPS_2D = 100
SEED_2D = 2026
CFL_2D = 0.5


FLOP_COUNTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle", "flop_counts.json")


def oracle_flops(path):
    """Algorithmic flops of one cell-stage on a path ("2d_euler_ng2_smooth",
    "1d_euler_troubled", ...): the oracle's operation count of that path (its
    sources compiled with a counting scalar), as stored in the table that
    oracle/count_flops.py writes (a data file: nothing of the oracle runs)."""
    with open(FLOP_COUNTS) as f:
        return json.load(f)["paths"][path]["cell_stage"]


def kernel_flops_per_cell_stage_2d(ng, ncomp=4):
    """The same count for the kernel's own formulation of a smooth 2D
    cell-stage (halo recomputation excluded): the linear p0 maps at the 4 ng
    interface and ng^2 interior points of every component (the nonzero
    coefficients of the generated maps over the 19 data: 228 for 2 Gauss
    points, 353 for 3; one multiply-add = 2 flops), the
    Lax-Friedrichs flux of each of the cell's own 2 ng interface points (Euler:
    two fluxes of 15 flops and 16 for the combination; Burgers: two u^2/2 and
    4), f and g at the interior points (Euler 2 x 15 + 16; Burgers 2 + 4), the
    right-hand-side sums (6 per quadrature point and component plus 10) and
    the Runge-Kutta combination (4 per moment).  Lower than the oracle's count
    (which also has the wave speeds, the KXRCF indicator and general
    polynomial evaluations); reported beside it."""
    nnz = 228 if ng == 2 else 353
    pt = 46 if ncomp == 4 else 8
    return (2 * ncomp * nnz + 2 * ng * pt + ng * ng * pt + ncomp * (6 * 3 * ng + 10)
            + 4 * 3 * ncomp)


def _time_2d(H, stream, cfg, dev, steps, warmup, nsteps, sampler=None):
    import torch
    h = H.hweno_create(cfg, stream.cuda_stream)
    try:
        def one_step():
            H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
            H.hweno_step(h, nsteps, -1.0, wait=False)
        for _ in range(warmup):
            one_step()
        H.hweno_step(h, 0, -1.0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        if sampler:
            sampler.__enter__()
        for k in range(steps):
            ev[k][0].record(stream)
            one_step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        H.hweno_step(h, 0, -1.0)
        st = H.hweno_stats(h)  # set_state resets the counters: the last timed step's
        return [a.elapsed_time(b) / 1e3 for a, b in ev], st, h
    except Exception:
        H.hweno_destroy(h)
        raise


def bench_euler2d(args, ngs=None, fp32_tflops=None):
    """2D Euler, 4096 x 4096 periodic [0, 10]^2, isentropic vortex plus seeded
    density modes, FP32, RK_STEPS_2D steps per bench step (state > L2), with
    the four-quadrant second run; one record per Gauss-point count."""
    import torch

    from paper_2002_08816_gb300 import hweno as H
    from paper_2002_08816_gb300 import workloads as W
    import __graft_entry__

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    burgers = args.workload == "burgers2d"
    ncomp = 1 if burgers else 4
    if ngs is None:
        ngs = [args.n_gauss or 2]
    if burgers:  # Example 3.9's data (0.5 + sin(pi (x + y)/2) on [0, 4]^2), past the shock
        u0 = W.burgers_sine_2d(NX2, NX2, npts=2).astype(np.float32)
    else:
        u0 = W.euler_vortex_modes_2d(NX2, NX2, seed=SEED_2D + rank, npts=2).astype(np.float32)
    dev = torch.from_numpy(u0).to("cuda")
    host_in = torch.from_numpy(u0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    hbm, peak_kind = peaks()
    if fp32_tflops is None:
        ap_ = alu_peaks()
        fp32_tflops = max(ap_["fp32_tflops"], ap_["fp32_packed_tflops"])
    cells = NX2 * NX2 * 3 * RK_STEPS_2D
    out = {}
    for ng in ngs:
        if burgers:
            cfg = H.make_config(2, H.HWENO_BURGERS, NX2, NX2, x0=0.0, x1=4.0, y0=0.0, y1=4.0,
                                bc=H.HWENO_BC_PERIODIC, cfl=0.6, precision=H.HWENO_FP32,
                                n_gauss=ng)
        else:
            cfg = H.make_config(2, H.HWENO_EULER, NX2, NX2, x0=0.0, x1=10.0, y0=0.0, y1=10.0,
                                bc=H.HWENO_BC_PERIODIC, cfl=CFL_2D, precision=H.HWENO_FP32,
                                n_gauss=ng)
        sampler = ClockSampler(local)
        ms, st, h = _time_2d(H, stream, cfg, dev, args.steps, args.warmup, RK_STEPS_2D, sampler)
        try:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            H.hweno_set_state(h, host_in.data_ptr(), H.HWENO_FP32, False)
            H.hweno_step(h, RK_STEPS_2D, -1.0, wait=False)
            H.hweno_get_state(h, host_out.data_ptr(), H.HWENO_FP32, False)
            b.record(stream)
            b.synchronize()
            e2e_s = a.elapsed_time(b) / 1e3
        finally:
            H.hweno_destroy(h)
        tot = sum(ms)
        stage_s = tot / (args.steps * 3 * RK_STEPS_2D)
        fpc = oracle_flops("2d_%s_ng%d_smooth" % ("burgers" if burgers else "euler", ng))
        fpk = kernel_flops_per_cell_stage_2d(ng, ncomp)
        flops = fpc * NX2 * NX2
        byts = (8 * 3 * 4 * ncomp / 3) * NX2 * NX2  # 8S/3, S = 3 moments x ncomp x 4 B
        t_alu = flops / (fp32_tflops * 1e12)
        t_hbm = byts / (hbm * 1e9)
        traffic = TRAFFIC_2D_NG2 if (ng == 2 and not burgers) else None
        if t_alu >= t_hbm:
            roof = {"bound": "alu", "achieved": flops / stage_s / 1e12, "peak": fp32_tflops,
                    "unit": "TFLOP/s", "frac": t_alu / stage_s, "traffic": traffic,
                    "flops_per_cell_stage": fpc,
                    "frac_kernel_count": fpk * NX2 * NX2 / (fp32_tflops * 1e12) / stage_s,
                    "note": "peak = measured FP32 FMA throughput (hweno_fma_peak, the larger of "
                            "the scalar and the packed fma.rn.f32x2 figures); %.0f flops per "
                            "smooth cell-stage counted on the oracle (oracle/flop_counts.json); "
                            "frac_kernel_count: the kernel's own %d" % (fpc, fpk)}
        else:
            roof = {"bound": "hbm", "achieved": byts / stage_s / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": t_hbm / stage_s, "traffic": traffic, "note": "peak %s" % peak_kind}
        roof["kernel"] = "stage2d_kernel<float,%d,%d>" % (ncomp, ng)
        rec = {
            "metric": METRIC, "value": cells * args.steps / tot, "unit": UNIT,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "stage_ms": stage_s * 1e3, "dtype": "f32",
            "config": {"workload": ("2D Burgers 4096x4096 periodic on [0,4]^2, 0.5 + sin(pi "
                                    "(x+y)/2) (Example 3.3/3.9 data), %d RK3 steps, %d Gauss "
                                    "points, CFL 0.6, FP32" % (RK_STEPS_2D, ng)) if burgers else
                                   ("2D Euler 4096x4096 periodic, vortex + 8 density modes, %d "
                                    "RK3 steps, %d Gauss points, CFL %.1f, FP32"
                                    % (RK_STEPS_2D, ng, CFL_2D)),
                       "seed": SEED_2D, "l2": "state (%d MB) larger than L2" % (u0.nbytes // 10 ** 6)},
            "troubled_frac": st["troubled"] / float(cells),
            "roofline": roof,
            "e2e": {"value": cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": host_in.numel() * 4,
                    "d2h_bytes_per_step": host_in.numel() * 4},
            "gpu_launches": args.steps * (4 * RK_STEPS_2D + 4),
            "clocks": sampler.summary(),
        }
        if not burgers and ng == ngs[0]:
            # the workload's second run: four constant quadrants drawn from the
            # seed (shocks and troubled cells), same grid, steps and CFL
            uq = W.euler_quadrants_2d(NX2, NX2, seed=SEED_2D + rank, npts=2).astype(np.float32)
            devq = torch.from_numpy(uq).to("cuda")
            del uq
            msq, stq, hq = _time_2d(H, stream, cfg, devq, max(1, args.steps - 1), 1, RK_STEPS_2D)
            H.hweno_destroy(hq)
            del devq
            q_s = sum(msq) / len(msq)
            rec["quadrants"] = {
                "value": cells / q_s, "ms_per_step": 1e3 * q_s,
                "stage_ms": 1e3 * q_s / (3 * RK_STEPS_2D),
                "troubled_frac": stq["troubled"] / float(cells),
                "roofline": {"bound": roof["bound"], "frac": roof["frac"] * (tot / args.steps) / q_s,
                             "note": "the smooth roofline's fraction at this run's time"},
                "data": "four constant quadrants (rho, u, v, p) drawn from the seed"}
        if not burgers:
            # the same vortex run with the float-pair averages (HWENO_FP32C)
            cfg.precision = H.HWENO_FP32C
            msc, _, hc = _time_2d(H, stream, cfg, dev, max(1, args.steps - 1), 1, RK_STEPS_2D)
            H.hweno_destroy(hc)
            cfg.precision = H.HWENO_FP32
            c_s = sum(msc) / len(msc)
            rec["fp32c"] = {"value": cells / c_s, "ms_per_step": 1e3 * c_s,
                            "stage_ms": 1e3 * c_s / (3 * RK_STEPS_2D),
                            "roofline": {"bound": roof["bound"],
                                         "frac": roof["frac"] * (tot / args.steps) / c_s,
                                         "note": "the FP32 roofline's fraction at this run's time "
                                                 "(the same algorithmic flops)"}}
        out["ng%d" % ng] = rec
    return out


# ----------------------------------------------------------------------------- adjoint workload

NX_ADJ = 1024
STEPS_ADJ = 200
EVERY_ADJ = 20
SEED_ADJ = 4242


def bench_adjoint2d(args, data="vortex"):
    """Gradient of sum(rho^2) after STEPS_ADJ steps with respect to the initial
    moments: 2D Euler 1024 x 1024 periodic [0, 10]^2, vortex plus density
    modes (or, data="quadrants", four constant quadrants drawn from the seed,
    whose shocks keep troubled cells in the tape), FP32, forward with the tape
    (checkpoint every EVERY_ADJ steps), then the checkpointed adjoint.  Reports
    forward, backward and their ratio."""
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
    if data == "quadrants":
        u0 = W.euler_quadrants_2d(n, n, seed=SEED_ADJ + rank).astype(np.float32)
    else:
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
    sampler.__exit__(None, None, None)
    troubled = H.hweno_stats(h)["troubled"]
    H.hweno_destroy(h)
    t_f, t_b = statistics.median(tf), statistics.median(tb)
    cells = n * n * 3 * STEPS_ADJ
    return {
        "metric": "cell-stages/s of forward + adjoint (gradient of sum rho^2)",
        "value": cells / (t_f + t_b), "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * (t_f + t_b), "dtype": "f32",
        "config": {"workload": "adjoint: 2D Euler 1024x1024 periodic, %s, "
                               "loss sum(rho^2) after %d RK3 steps, checkpoint every %d, "
                               "%d Gauss points, FP32"
                               % ("four constant quadrants (shocks)" if data == "quadrants"
                                  else "vortex + 8 density modes", STEPS_ADJ, EVERY_ADJ, ng),
                   "seed": SEED_ADJ, "l2": "state 50 MB, tape and segment states > L2"},
        "forward_ms": t_f * 1e3, "backward_ms": t_b * 1e3,
        "adjoint_over_forward": t_b / t_f,
        "forward_cell_stages_per_s": cells / t_f,
        "troubled_frac_forward": troubled / float(cells),
        "fd_check": "tests/test_gpu_adjoint2d.py::test_backward_matches_finite_differences_64 "
                    "(64x64, 16 directions, within 1e-4 in FP32 and FP64)",
        "clocks": sampler.summary(),
        # forward and recomputed stages with their dt kernels, two adjoint
        # kernels and a fix-up pass per stage, one wave-speed launch per
        # segment, and the state conversions and resets
        "gpu_launches": args.steps * (3 * STEPS_ADJ * 2 + STEPS_ADJ * 2 + 9 * STEPS_ADJ
                                      + STEPS_ADJ // EVERY_ADJ + 6),
    }


# ----------------------------------------------------------------------------- batched 1D workload

N_BATCH = 512
RK_STEPS_BATCH = 500
SEED_BATCH = 77


def bench_batch1d(args):
    """512 independent 1D Euler instances, cell counts log-uniform in
    [256, 16384], two-state data, FP32, RK_STEPS_BATCH steps each, advanced in
    shared launches; against one handle per instance for all 512 instances."""
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
    # one handle per instance, all 512 of them, each in its own CUDA graphs
    handles = []
    try:
        for b in range(N_BATCH):
            c1 = H.make_config(1, H.HWENO_EULER, sizes[b], x0=0.0, x1=1.0, bc=H.HWENO_BC_OUTFLOW,
                               cfl=CFL, precision=H.HWENO_FP32)
            hb = H.hweno_create(c1, stream.cuda_stream)
            handles.append((hb, torch.from_numpy(states[b]).to("cuda")))
        for hb, d in handles:  # warm-up: builds both graphs of every handle
            H.hweno_set_state(hb, d.data_ptr(), H.HWENO_FP32, True)
            H.hweno_step(hb, 33, -1.0, wait=False)
        torch.cuda.synchronize()
        flush.fill_(-1.0)
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for hb, d in handles:
            H.hweno_set_state(hb, d.data_ptr(), H.HWENO_FP32, True)
            H.hweno_step(hb, RK_STEPS_BATCH, -1.0, wait=False)
        b2.record(stream)
        b2.synchronize()
        per_inst_s = a.elapsed_time(b2) / 1e3
        for hb, _ in handles:
            H.hweno_step(hb, 0, -1.0)  # status check
    finally:
        for hb, _ in handles:
            H.hweno_destroy(hb)
    value = cells * 3 * RK_STEPS_BATCH * args.steps / tot
    hbm, peak_kind = peaks()
    stage_s = tot / (args.steps * 3 * RK_STEPS_BATCH)
    achieved = BYTES_PER_CELL_STAGE["fp32"] * cells / stage_s / 1e9
    launch = LAUNCH_KIND[choice[1]]
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "dtype": "f32",
        "config": {"workload": "batched 1D Euler: 512 instances, cells log-uniform in "
                               "[256, 16384] (%d cells), two-state data, %d RK3 steps each, "
                               "CFL %.1f, FP32, all instances in shared launches"
                               % (cells, RK_STEPS_BATCH, CFL),
                   "seed": SEED_BATCH, "l2": "flushed (512 MiB write) between timed steps"},
        "per_instance": {"ms_per_step": 1e3 * per_inst_s,
                         "value": cells * 3 * RK_STEPS_BATCH / per_inst_s,
                         "how": "one handle per instance for all 512 instances (CUDA graphs of 32 "
                                "steps and of one step), the same steps, one stream"},
        "speedup_vs_per_instance": per_inst_s / (tot / args.steps),
        "execution": {"threads_per_cta": choice[0], "launch": launch,
                      "chosen_by": "hweno_autotune"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": TRAFFIC_BATCH_FP32.get((choice[0], launch)),
                     "kernel": "%s<float,3,batch,%d threads>" % (KERNEL_OF_LAUNCH[launch],
                                                                choice[0]),
                     "note": "avg stage time = timed region (set_state included) / %d stages; "
                             "the %d MB state fits in L2; peak %s"
                             % (3 * RK_STEPS_BATCH, cells * 24 // 10 ** 6, peak_kind)},
        "gpu_launches": args.steps * ((3 * RK_STEPS_BATCH if launch == "per-stage graphs" else 1) + 5),
        "clocks": sampler.summary(),
    }


# ----------------------------------------------------------------------------- troubled-cell path

RK_STEPS_TROUBLED = 200


def bench_troubled1d(args):
    """The headline kernel on data with a paper-like share of troubled cells:
    the Lax problem's states repeated every 800 cells over 65536 cells
    (periodic), FP32, RK_STEPS_TROUBLED steps per bench step."""
    import torch

    from paper_2002_08816_gb300 import hweno as H
    from paper_2002_08816_gb300 import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    u0 = W.euler_lax_tiled_1d(NX).astype(np.float32)
    cfg = H.make_config(1, H.HWENO_EULER, NX, x0=0.0, x1=1.0, bc=H.HWENO_BC_PERIODIC, cfl=CFL,
                        precision=H.HWENO_FP32)
    h = H.hweno_create(cfg, stream.cuda_stream)
    dev = torch.from_numpy(u0).to("cuda")
    try:
        H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
        choice = H.hweno_autotune(h, 50)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
            H.hweno_step(h, RK_STEPS_TROUBLED, -1.0, wait=False)
        H.hweno_step(h, 0, -1.0)
        ms = []
        sampler = ClockSampler(0)
        sampler.__enter__()
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            H.hweno_set_state(h, dev.data_ptr(), H.HWENO_FP32, True)
            H.hweno_step(h, RK_STEPS_TROUBLED, -1.0, wait=False)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        sampler.__exit__(None, None, None)
        H.hweno_step(h, 0, -1.0)
        st = H.hweno_stats(h)
    finally:
        H.hweno_destroy(h)
    tot = sum(ms) / 1e3
    cells = NX * 3 * RK_STEPS_TROUBLED
    frac = st["troubled"] / float(cells)
    stage_s = tot / (args.steps * 3 * RK_STEPS_TROUBLED)
    hbm, peak_kind = peaks()
    achieved = BYTES_PER_CELL_STAGE["fp32"] * NX / stage_s / 1e9
    smooth, troubled = oracle_flops("1d_euler_smooth"), oracle_flops("1d_euler_troubled")
    launch = LAUNCH_KIND[choice[1]]
    return {
        "metric": METRIC, "value": cells * args.steps / tot, "unit": UNIT, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "dtype": "f32",
        "stage_us": stage_s * 1e6,
        "config": {"workload": "1D Euler, the Lax problem's states repeated every 800 cells "
                               "over 65536 cells, periodic, %d RK3 steps, CFL %.1f, FP32"
                               % (RK_STEPS_TROUBLED, CFL),
                   "l2": "flushed (512 MiB write) between timed steps"},
        "troubled_frac": frac,
        "paper_troubled_frac": "Examples 3.6-3.8: 13.41 %, 3.54 %, 13.94 %",
        "execution": {"threads_per_cta": choice[0], "launch": launch,
                      "chosen_by": "hweno_autotune"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": TRAFFIC_TROUBLED_1D.get((choice[0], launch)),
                     "kernel": "%s<float,3,%d threads>" % (KERNEL_OF_LAUNCH[launch], choice[0]),
                     "flops_per_cell_stage": smooth + frac * (troubled - smooth),
                     "note": "64 B per cell-stage; flops counted on the oracle "
                             "(oracle/flop_counts.json): %.0f per smooth and %.0f per troubled "
                             "cell-stage at the measured share; peak %s"
                             % (smooth, troubled, peak_kind)},
        "gpu_launches": args.steps * ((3 * RK_STEPS_TROUBLED if launch == "per-stage graphs" else 1) + 4),
        "clocks": sampler.summary(),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hweno", choices=["hweno", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the other workloads' sub-records of the default run")
    ap.add_argument("--workload", default="euler1d",
                    choices=["euler1d", "euler2d", "burgers2d", "batch1d", "adjoint2d",
                             "adjoint2d_quadrants", "troubled1d"],
                    help="euler1d: the headline 65536-cell 1D workload (with every other "
                         "workload as a sub-record at one GPU); the others alone")
    ap.add_argument("--n-gauss", type=int, default=None, choices=[2, 3],
                    help="Gauss points per direction (2D): default 2 for euler2d (its "
                         "configuration), 3 for adjoint2d (the paper's)")
    args = ap.parse_args()
    if args.impl == "reference":
        line = bench_reference(args)
    elif args.workload == "euler1d":
        line = bench_hweno(args)
        ws, _, _ = dist_env()
        if line is not None and ws == 1 and not args.headline_only:
            sub = copy.copy(args)
            # every sub-record takes the command's warm-up count (>= 3) and up
            # to 2 timed steps
            sub.steps, sub.warmup = max(1, min(args.steps, 2)), max(3, args.warmup)
            ap_ = alu_peaks()
            line["alu_peaks"] = ap_
            # the FP64 path is bound by GB300's FP64 pipe (1/64 of FP32): its
            # arithmetic roofline, the oracle's flops per cell-stage at the
            # run's troubled share over the measured FP64 FMA peak
            tf = line["troubled_frac"]
            fl64 = ((1.0 - tf) * oracle_flops("1d_euler_smooth")
                    + tf * oracle_flops("1d_euler_troubled"))
            ach64 = line["fp64"]["value"] * fl64 / 1e12
            line["fp64"]["roofline"] = {
                "bound": "alu", "unit": "TFLOP/s", "peak": ap_["fp64_tflops"], "achieved": ach64,
                "frac": ach64 / ap_["fp64_tflops"], "traffic": None,
                "flops_per_cell_stage": fl64,
                "note": "oracle op count per cell-stage (oracle/flop_counts.json) at the FP32 "
                        "run's troubled share x cell-stages/s; peak = measured FP64 FMA "
                        "throughput (hweno_fma_peak)"}
            wl = {}

            def sub_record(name, fn, *a, **k):
                # a failing sub-record is reported, it does not void the headline
                try:
                    wl[name] = fn(*a, **k)
                except Exception as exc:  # noqa: BLE001
                    wl[name] = {"error": "%s: %s" % (type(exc).__name__, str(exc)[:300])}
            sub.workload, sub.n_gauss = "euler2d", None
            sub_record("euler2d", bench_euler2d, sub, ngs=[2, 3],
                       fp32_tflops=max(ap_["fp32_tflops"], ap_["fp32_packed_tflops"]))
            sub.workload = "batch1d"
            sub_record("batch1d", bench_batch1d, sub)
            sub.workload = "adjoint2d"
            sub_record("adjoint2d", bench_adjoint2d, sub)
            sub_record("adjoint2d_quadrants", bench_adjoint2d, sub, data="quadrants")
            sub.workload = "troubled1d"
            sub_record("troubled1d", bench_troubled1d, sub)
            line["workloads"] = wl
    elif args.workload in ("euler2d", "burgers2d"):
        line = bench_euler2d(args)
    elif args.workload == "batch1d":
        line = bench_batch1d(args)
    elif args.workload == "adjoint2d":
        line = bench_adjoint2d(args)
    elif args.workload == "adjoint2d_quadrants":
        line = bench_adjoint2d(args, data="quadrants")
    else:
        line = bench_troubled1d(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
