#!/usr/bin/env python3
"""Throughput of the fused D2V16 DBM step on GB300.

Default workload: the Kelvin-Helmholtz shear layer on 4096 x 4096 cells with
2 species, f stored and stepped in FP32 (the largest single-grid
configuration), synthetic seeded initial fields, one fused kernel launch
per time step.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--workload kh4096|reactive|sod] [--precision fp32|fp64]

N > 1 runs under torchrun: every rank steps its own replica of the grid
(independent problems, no data-path collective) and the value is the sum of
all ranks' updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2V16 species-cell updates/s and HBM-roofline %, FP32 vs FP64; serve p50/p99"
UNIT = "species-cell updates/s"
BYTES_PER_UPDATE = {"fp64": 256, "fp32": 128}
FALLBACK_HBM_GBS = 6800.0
# The FP64 step (oracle operation order, no fused multiply-add) is bound by
# the FP64 pipe, not by HBM.  Its FP64 operations per species-cell update,
# from the ncu counts of one 1024 x 1024 two-species launch (DADD 85.8 +
# DMUL 80.1 + 2 x DFMA 46.2 flop per cycle over 12.24 ms at 2.06 GHz for
# 2.10 M updates), and the nominal FP64 peak of a GB300 (no measured FP64
# figure exists for this pool).
FP64_FLOPS_PER_UPDATE = 3107.0
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="kh4096", choices=["kh4096", "reactive", "sod", "batched", "serve",
                                                                    "precision_kh", "precision_reactive", "smooth"])
    ap.add_argument("--species", type=int, default=5,
                    help="species of the smooth workload (seeded smooth fields; five or more run the species-staged kernel)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16dev"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 and e2e side legs")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--grid", default=None, help="override the grid, e.g. 2048x1024 (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-steps", default="1000,10000", help="step counts drawn uniformly in lo,hi")
    ap.add_argument("--serve-sides", default="128,2048", help="sides drawn log-uniformly in lo,hi")
    ap.add_argument("--serve-load", type=float, default=0.8, help="arrival rate / measured capacity")
    ap.add_argument("--serve-qmax", type=int, default=128)
    ap.add_argument("--study-steps", type=int, default=None,
                    help="steps of a precision study (1000 for precision_kh, 20000 for precision_reactive)")
    return ap.parse_args()


def make_workload(name, grid=None, species=5):
    from paper_2006_15932_gb300 import workloads as W

    nx, ny = (int(v) for v in grid.lower().split("x")) if grid else (None, None)
    if name == "smooth":
        return W.random_smooth(nx or 1024, ny or 1024, species, seed=W.SEED)
    if name == "kh4096":
        return W.kh_shear_layer(nx or 4096, ny=ny)
    if name == "reactive":
        return W.reactive_premixed(nx or 1024, ny or 256)
    if name in ("batched", "serve"):  # the oracle's sample: one mid-size instance of the mix
        return W.shock_instance(nx or 288, W.SEED)
    return W.sod_tube(nx or 400, 2000)


def workload_config(pb, name, precision):
    return {
        "workload": {"kh4096": "kelvin_helmholtz_shear_layer", "reactive": "reactive_premixed_2d",
                     "sod": "sod_shock_tube", "batched": "batched_shock_and_reactive_instances",
                     "serve": "serve_poisson_request_mix", "smooth": "random_smooth_fields"}[name],
        "grid": [pb.nx, pb.ny],
        "species": pb.ns,
        "velocities": 16,
        "precision": precision,
        "reactive": pb.k_ov != 0.0,
        "boundary": ["periodic" if b == 0 else "outflow" for b in (pb.bc_x, pb.bc_y)],
        "state_bytes_per_buffer": int(pb.nx * pb.ny * pb.ns * 16 * bytes_per_update(precision, pb.ns) / 32),
        "l2_policy": "inputs larger than L2" if pb.nx * pb.ny * pb.ns * 64 > 129e6
        else "state fits in L2 (no flush)",
    }


def bytes_per_update(precision, ns):
    """Algorithmic HBM bytes per species-cell update: the 16 stored values
    read and written; BF16DEV adds the cell's S+3 float moments (read and
    written) shared by its S species."""
    if precision == "bf16dev":
        return 16 * 2 * 2 + 2 * (ns + 3) * 4 / ns
    return BYTES_PER_UPDATE[precision]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for rel in ("paper_2006_15932_gb300/csrc/dbm_step_impl.cuh", "paper_2006_15932_gb300/csrc/dbm_device.cuh",
                "paper_2006_15932_gb300/csrc/dbm_internal.h", "paper_2006_15932_gb300/csrc/dbm_step.cu"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def step_kernel_name(pb, precision, solver):
    """The step kernel dbm_step dispatches for this problem (DBM_KERNEL_AUTO);
    the TMA tile as the library reports it."""
    if precision == "fp64":
        return f"k_step_f64<{pb.ns}>"
    if precision == "bf16dev":
        return f"k_step_bf16<{pb.ns},32,16,2>"
    tx, ty, cw = solver.step_tile()
    if tx and cw == 2 and pb.ns >= 3:  # two cells per thread for three or more species: species-staged
        return f"k_step_staged<{pb.ns},{tx},{ty}>"
    if tx:
        return f"k_step_tma<{pb.ns},{tx},{ty},{cw}>"
    return f"k_step<{pb.ns}>"


def ncu_traffic(name, precision):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    key = f"{name}:{precision}"
    e = d.get(key)
    if not e or e.get("source_sha") != kernel_source_sha():
        return None
    return e.get("dram_bytes_per_launch")


def combine_ranks(ms_local, updates_per_rank, dist=None, device=None):
    """Whole-job throughput of replicas: every rank advanced its own
    independent problem by updates_per_rank species-cell updates; the job
    took as long as the slowest rank.  Returns (max ms over ranks, total
    updates of all ranks / that time)."""
    import torch

    ms = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_initialized():
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms_max = float(ms.item())
    return ms_max, updates_per_rank * world / (ms_max * 1e-3)


class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            # raw samples (the JSON line carries their summary)
            out_dir = os.environ.get("DBM_CLOCKS_DIR") or tempfile.gettempdir()
            os.makedirs(out_dir, exist_ok=True)
            self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and self.uuid not in parts[1]:
                continue
            try:
                sm.append(float(parts[2].split()[0]))
                smax.append(float(parts[3].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(pb_full, precision, seconds, one_core=True):
    """The FP64 oracle as it stands, on the host cores, over a bounded
    sample of the workload: a window of the same grid (same species,
    parameters and initial fields) stepped a few times."""
    import numpy as np

    from oracle import oracle as O
    from paper_2006_15932_gb300 import workloads as W

    nx = min(pb_full.nx, 512)
    ny = min(pb_full.ny, 256)
    x0 = (pb_full.nx - nx) // 2
    y0 = (pb_full.ny - ny) // 2
    pb = W.Problem(name=pb_full.name + "_window", nx=nx, ny=ny, species=pb_full.species, dx=pb_full.dx,
                   dy=pb_full.dy, dt=pb_full.dt, bc_x=pb_full.bc_x, bc_y=pb_full.bc_y, fuel=pb_full.fuel,
                   oxid=pb_full.oxid, k_ov=pb_full.k_ov, Ea_over_R=pb_full.Ea_over_R, Q=pb_full.Q,
                   accel=pb_full.accel, rho_s=pb_full.rho_s[:, y0:y0 + ny, x0:x0 + nx],
                   ux=pb_full.ux[y0:y0 + ny, x0:x0 + nx], uy=pb_full.uy[y0:y0 + ny, x0:x0 + nx],
                   T=pb_full.T[y0:y0 + ny, x0:x0 + nx])
    p = O.params_of(pb)
    f = O.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)

    def timed(budget):
        O.run(p, f, 1)  # start the OpenMP thread pool
        t0 = time.perf_counter()
        g, st = O.run(p, f, 1)
        per_step = max(time.perf_counter() - t0, 1e-6)
        steps = max(1, min(1000, int(budget / per_step)))
        t0 = time.perf_counter()
        _, st2 = O.run(p, g, steps)
        dt = time.perf_counter() - t0
        if st or st2:
            raise RuntimeError(f"oracle status {st}/{st2} on the CPU-baseline sample: the timing would be cut short")
        return steps, dt

    cores = O.set_threads(0)
    steps, dt = timed(seconds)
    window = f"{nx}x{ny} window of the {pb_full.nx}x{pb_full.ny} grid, {pb.ns} species"
    out = {"value": nx * ny * pb.ns * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{window}, {steps} FP64 steps in {dt:.1f} s (OpenMP over rows)"}
    if one_core and cores > 1:  # the same sample on one core, for a quarter of the time
        O.set_threads(1)
        try:
            s1, d1 = timed(seconds / 4)
        finally:
            O.set_threads(cores)
        out["one_core"] = {"value": nx * ny * pb.ns * s1 / d1, "unit": UNIT, "cores": 1,
                           "sample": f"{window}, {s1} FP64 steps in {d1:.1f} s"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pb = make_workload(args.workload, args.grid, args.species)
    cfg = workload_config(pb, args.workload, args.precision)
    # each "step" of the reference arm is a bounded sample of the workload
    per = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(pb, args.precision, per / 4, one_core=False)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(pb, args.precision, per, one_core=False))
    wall = time.perf_counter() - t0
    value = statistics.median(v["value"] for v in vals)
    cb = dict(vals[-1])
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serve_study(D, dev, mix, load, qmax, subset_n):
    """Continuous batching on a request mix, measured three ways.

    1. capacity: the mix arriving all at once, served (species-cell updates
       per second over the makespan);
    2. the served run: Poisson arrivals at `load` x capacity; p50 / p99
       latency (arrival -> conserved totals on the host) and throughput;
    3. the baseline, on a stated subset (the `subset_n` requests with the
       fewest updates, all arriving at once): the same requests served with
       continuous batching (FP32), solved one at a time in FP64 and in FP32
       (real solves, serve.run_sequential); throughputs, latencies, and the
       served results' largest relative L-inf distance from the FP64 solves
       (the accuracy at which the throughputs are compared)."""
    import dataclasses

    import torch

    from paper_2006_15932_gb300 import serve as SV
    from paper_2006_15932_gb300 import workloads as W

    SV.Server(device=dev, qmax=qmax).run(mix[:4])  # warm-up: kernels, allocator
    cap = SV.summarize(SV.Server(device=dev, qmax=qmax).run(mix))["throughput"]
    mean_units = sum(q.units for q in mix) / len(mix)
    rate = load * cap / mean_units
    timed = W.poisson_arrivals(mix, rate)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    srv = SV.Server(device=dev, qmax=qmax)
    res = srv.run(timed)
    clk = clocks.stop()
    if any(r.status for r in res):
        raise SystemExit("health flag raised while serving")
    summ = SV.summarize(res)

    sub = [dataclasses.replace(q, arrival=0.0) for q in sorted(mix, key=lambda q: q.units)[:subset_n]]
    served = {r.rid: r for r in SV.Server(device=dev, qmax=qmax, keep_f=True).run(sub)}
    seq64 = {r.rid: r for r in SV.run_sequential(sub, "fp64", device=dev, keep_f=True)}
    seq32 = {r.rid: r for r in SV.run_sequential(sub, "fp32", device=dev)}
    if any(r.status for r in list(served.values()) + list(seq64.values()) + list(seq32.values())):
        raise SystemExit("health flag raised in the serving baseline")
    acc = max(float(np.max(np.abs(served[k].f - seq64[k].f)) / np.max(np.abs(seq64[k].f))) for k in served)

    def brief(results):
        d = SV.summarize(list(results))
        return {k: d[k] for k in ("p50_s", "p99_s", "mean_s", "makespan_s", "throughput")}

    return {
        "capacity_units_per_s": cap, "arrival_rate_per_s": rate, "load": load, "requests": len(mix),
        "p50_s": summ["p50_s"], "p99_s": summ["p99_s"], "mean_s": summ["mean_s"],
        "makespan_s": summ["makespan_s"], "throughput": summ["throughput"], "units": summ["units"],
        "hbm_budget_bytes": srv.adm.budget, "admitted_peak_bytes": srv.adm.peak,
        "batch_rebuilds": sum(g.rebuilds for g in srv.groups.values()), "quanta": srv.launch_quanta,
        "batch_config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in srv.config.items()},
        "clocks": clk,
        "baseline": {
            "subset": f"the {len(sub)} requests of the mix with the fewest updates, all arriving at t = 0",
            "units": sum(q.units for q in sub),
            "served_fp32": brief(served.values()),
            "sequential_fp64": brief(seq64.values()),
            "sequential_fp32": brief(seq32.values()),
            "served_vs_fp64_rel_linf_f": acc,
            "how": "sequential = first come, first served, one request at a time, each a plain single-problem "
                   "solve (real runs, serve.run_sequential)",
        },
    }


def run_serve(args, D, dev):
    """Serving (the request-mix configuration): Poisson arrivals at a
    fraction of the measured capacity, continuous batching; p50/p99 latency
    and throughput; sequential FP64 and FP32 solves of a stated subset of the
    mix as the measured baseline, and of the whole mix as an extrapolation
    from rates measured here."""
    import torch

    from paper_2006_15932_gb300 import serve as SV
    from paper_2006_15932_gb300 import workloads as W

    s_lo, s_hi = (int(v) for v in args.serve_sides.split(","))
    n_lo, n_hi = (int(v) for v in args.serve_steps.split(","))
    specs = W.serving_requests(args.serve_requests, lo=s_lo, hi=s_hi, steps=(n_lo, n_hi))
    st = serve_study(D, dev, specs, args.serve_load, args.serve_qmax, subset_n=8)

    # extrapolation to the whole mix: FIFO queue with service times from the
    # FP64 and unbatched FP32 rates measured per species count on a 512 x 512
    # shock tube (FP64 is ALU-bound, so its rate hardly depends on the size)
    def rate_of(precision, ns, steps):
        spec = W.RequestSpec(rid=0, kind="shock", L=512, ns=ns, seed=1, nsteps=steps)
        stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(stream):
            s = D.Solver(W.request_problem(spec), precision, device=dev)
            s.set_state(*W.request_fields(spec, dev))
            s.step(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        return 512 * 512 * ns * steps / (ms * 1e-3)

    nss = sorted({q.ns for q in specs})
    r64 = {ns: rate_of("fp64", ns, 4) for ns in nss}
    r32 = {ns: rate_of("fp32", ns, 200) for ns in nss}
    timed = W.poisson_arrivals(specs, st["arrival_rate_per_s"])
    peak, peak_kind = measured_peaks()
    bpu = BYTES_PER_UPDATE["fp32"]
    cfg = {"workload": "serve_poisson_request_mix", "requests": len(specs), "sides": [s_lo, s_hi],
           "side_distribution": "log-uniform", "species": nss, "reactive_fraction": 0.5,
           "steps": [n_lo, n_hi], "precision": "fp32", "arrival_rate_per_s": st["arrival_rate_per_s"],
           "load": args.serve_load, "capacity_units_per_s": st["capacity_units_per_s"], "qmax": args.serve_qmax,
           "batch_config": st["batch_config"], "l2_policy": "inputs larger than L2"}
    clk = st.pop("clocks")
    line = {"metric": METRIC, "value": st["throughput"], "unit": UNIT, "n_gpus": 1, "steps": len(specs),
            "warmup": 4, "ms_per_step": 1e3 * st["makespan_s"] / len(specs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded request mix, Poisson arrivals)", "config": cfg, "serve": st,
            "extrapolated_sequential": {
                "fp64": dict(SV.simulate_sequential(timed, r64), rate_by_species=r64),
                "fp32_unbatched": dict(SV.simulate_sequential(timed, r32), rate_by_species=r32),
                "how": "not a run: FIFO queue over the whole mix with service time = updates / rate measured on "
                       "a 512x512 tube per species count"},
            "clocks": clk, "e2e": {"value": st["throughput"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                   "d2h_bytes_per_step": 8 * (max(nss) + 4)},
            "roofline": {"bound": "hbm", "achieved": st["throughput"] * bpu / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": st["throughput"] * bpu / 1e9 / peak, "traffic": None,
                         "kernel": "all step kernels of the run (whole-run average)",
                         "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}}
    print(json.dumps(line), flush=True)
    return 0


# Arithmetic variants of the precision studies: name -> (precision, options)
STUDY_VARIANTS = {
    "fp64": ("fp64", {}),
    "fp32": ("fp32", {}),
    "fp32_thermo64": ("fp32", {"thermo": "fp64"}),
    "fp32_stochastic": ("fp32", {"rounding": "stochastic"}),
    "fp32_thermo64_stochastic": ("fp32", {"thermo": "fp64", "rounding": "stochastic"}),
    "bf16dev": ("bf16dev", {}),
}


def run_precision(args, D, dev):
    """Precision study: the same initial state advanced in FP64 and in the
    float variants (FP32 with its thermo and rounding options, BF16DEV where
    its scope allows); relative L2 and L-infinity errors of the mixture
    fields against FP64 at checkpoints, each variant's drift of the conserved
    totals at the same checkpoints, and the step time of each variant."""
    import torch

    from paper_2006_15932_gb300 import workloads as W

    if args.workload == "precision_kh":
        nx, ny = (int(v) for v in (args.grid or "4096x4096").lower().split("x"))
        pb = W.kh_shear_layer(nx, ny=ny)
        total = args.study_steps or 1000
        precs = ["fp64", "fp32", "fp32_thermo64", "fp32_stochastic", "bf16dev"]
        checkpoints = 4
    else:
        nx, ny = (int(v) for v in (args.grid or "1024x256").lower().split("x"))
        pb = W.reactive_premixed(nx, ny)
        total = args.study_steps or 20000
        precs = ["fp64", "fp32", "fp32_thermo64", "fp32_stochastic", "fp32_thermo64_stochastic"]
        checkpoints = 10
    st = torch.cuda.Stream(device=dev)
    sols = {}
    with torch.cuda.stream(st):
        for p in precs:
            prec, opts = STUDY_VARIANTS[p]
            sols[p] = D.Solver(pb, prec, device=dev, **opts)
            sols[p].set_state()
        cons0 = {p: sols[p].conservation().cpu().numpy() for p in precs}
    S = pb.ns
    names = ["rho", "ux", "uy", "T"]
    rows = {"rho": 4 * S, "ux": 4 * S + 1, "uy": 4 * S + 2, "T": 4 * S + 3}

    def drift_of(c1, c0):
        mass0 = float(sum(abs(c0[:S])))
        e_scale = abs(float(c0[S + 2])) + abs(float(c0[S + 3]))
        return {"mass": float((sum(c1[:S]) - sum(c0[:S])) / mass0),
                "momentum_x": float((c1[S] - c0[S]) / mass0),
                "momentum_y": float((c1[S + 1] - c0[S + 1]) / mass0),
                "energy_plus_bound_heat": float(((c1[S + 2] + c1[S + 3]) - (c0[S + 2] + c0[S + 3])) / e_scale)}

    # velocity errors are measured against the velocity scale of the run
    # (max |u| of the FP64 field, at least the sound speed 1), not against a
    # field that may vanish
    curve = []
    per = total // checkpoints
    done = 0
    t_step = {p: 0.0 for p in precs}
    while done < total:
        n = min(per, total - done)
        mom = {}
        with torch.cuda.stream(st):
            for p in precs:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                sols[p].step(n)
                e1.record(st)
                e1.synchronize()
                t_step[p] += e0.elapsed_time(e1) * 1e-3
                mom[p] = sols[p].moments()
            cons = {p: sols[p].conservation().cpu().numpy() for p in precs}
        st.synchronize()
        done += n
        ref = mom["fp64"]
        entry = {"step": done, "drift": {p: drift_of(cons[p], cons0[p]) for p in precs}}
        for p in precs[1:]:
            errs = {}
            for nm in names:
                a, b = mom[p][rows[nm]], ref[rows[nm]]
                scale = torch.max(torch.abs(b))
                if nm in ("ux", "uy"):
                    scale = torch.maximum(torch.max(torch.abs(ref[rows["ux"]]).max(), torch.abs(ref[rows["uy"]]).max()),
                                          torch.tensor(1.0, dtype=torch.float64, device=dev))
                d = a - b
                errs[nm] = {"rel_linf": float(torch.max(torch.abs(d)) / scale),
                            "rel_l2": float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(b)
                                            if nm not in ("ux", "uy") else
                                            torch.linalg.vector_norm(d) / (scale * math.sqrt(d.numel())))}
            entry[p] = errs
        curve.append(entry)
        del mom, ref
    for p in precs:
        rc, bits = sols[p].status()
        if rc != 0:
            raise SystemExit(f"health flag raised in {p}: bits={bits}")
        sols[p].close()
    final = curve[-1]["drift"]
    line = {"study": args.workload, "grid": [pb.nx, pb.ny], "species": S, "steps": total,
            "boundary": ["periodic" if b == 0 else "outflow" for b in (pb.bc_x, pb.bc_y)],
            "reactive": pb.k_ov != 0.0,
            "variants": {p: {"precision": STUDY_VARIANTS[p][0], **STUDY_VARIANTS[p][1]} for p in precs},
            "updates_per_s": {p: pb.nx * pb.ny * S * total / t_step[p] for p in precs},
            "error_vs_fp64": curve, "conservation_drift": final,
            "conservation_drift_minus_fp64": {p: {k: final[p][k] - final["fp64"][k] for k in final[p]}
                                              for p in precs},
            "norms": "rel_linf = max|a-b| / max|b|, rel_l2 = ||a-b|| / ||b||; for u_x, u_y the scale is "
                     "max(max|u|, 1) (and rms of that scale for L2); drift = (total(t) - total(0)) / scale, "
                     "signed; the energy total includes the heat bound in the fuel"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2006_15932_gb300 import build as B
    from paper_2006_15932_gb300 import dbm as D

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "serve":
        B.build()
        D.load()
        return run_serve(args, D, dev) if rank == 0 else 0
    if args.workload.startswith("precision"):
        B.build()
        D.load()
        return run_precision(args, D, dev) if rank == 0 else 0
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    D.load()

    stream = torch.cuda.Stream(device=dev)
    if args.workload == "batched":
        from paper_2006_15932_gb300 import workloads as W

        pbs = W.batched_instances()
        pb = pbs[0]
        cfg = {"workload": "batched_shock_and_reactive_instances", "instances": len(pbs),
               "grids": "square, sides uniform in [64, 512] (seeded)", "species": 2, "velocities": 16,
               "precision": args.precision, "cells": sum(q.nx * q.ny for q in pbs),
               "l2_policy": "inputs larger than L2",
               "launch": "one launch per step over all instances' tiles, pairs of steps replayed from a CUDA graph"}
        solvers = [D.Solver(q, args.precision, device=dev, stream=stream) for q in pbs]
        for s_ in solvers:
            s_.set_state()
        batch = D.Batch(solvers, stream=stream, tune=True)
        info = batch.info()
        cfg["tile"] = list(info["tile"])
        cfg["ctas_per_launch"] = info["ctas"]
        cfg["tiles_per_step"] = info["tiles"]
        cfg["batch_config"] = {k: (list(v) if isinstance(v, tuple) else v) for k, v in batch.config().items()}
        units = sum(q.nx * q.ny * q.ns for q in pbs)
        per_call = 2  # one graph replay = two steps

        def advance(n):
            batch.step(n)

        solver = solvers[0]
    else:
        pb = make_workload(args.workload, args.grid, args.species)
        cfg = workload_config(pb, args.workload, args.precision)
        solver = D.Solver(pb, args.precision, device=dev, stream=stream)
        solver.set_state()
        units = pb.nx * pb.ny * pb.ns
        per_call = 1

        def advance(n):
            solver.step(n)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            advance(per_call)
    torch.cuda.synchronize(dev)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    K = max(per_call, args.steps // per_call * per_call)
    calls = K // per_call
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(calls + 1)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.25)  # let the sampler start
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(calls):
            advance(per_call)
            ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    per_launch = [ev[k].elapsed_time(ev[k + 1]) / per_call for k in range(calls)]
    ms_total = ev[0].elapsed_time(ev[calls])
    for s_ in (solvers if args.workload == "batched" else [solver]):
        rc, bits = s_.status()
        if rc != 0:
            raise SystemExit(f"health flag raised during the benchmark: rc={rc} bits={bits}")
    updates_per_rank = units * K
    ms_max, value = combine_ranks(ms_total, updates_per_rank, dist, dev)

    peak, peak_kind = measured_peaks()
    bpu = bytes_per_update(args.precision, pb.ns)
    avg_launch_ms = statistics.mean(per_launch)
    bytes_per_launch = units * bpu
    achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
    traffic = ncu_traffic(args.workload, args.precision)
    if args.precision == "fp64":
        tflops = value * FP64_FLOPS_PER_UPDATE / 1e12
        roofline = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None,
                    "peak_source": "nominal GB300 FP64 (no measured FP64 peak); the kernel keeps the oracle's "
                                   "operation order, so separate adds and multiplies fill the FP64 pipe "
                                   "(84.5 % busy per ncu) at half the flops of fused multiply-adds",
                    "kernel": step_kernel_name(pb, args.precision, solver), "flops_per_update": FP64_FLOPS_PER_UPDATE,
                    "hbm_gbs": achieved, "median_launch_ms": statistics.median(per_launch)}
    else:
        roofline = None
    roofline = roofline or {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "kernel": step_kernel_name(pb, args.precision, solver) if args.workload != "batched"
                else f"k_step_batch<{pb.ns},{cfg['tile'][0]},{cfg['tile'][1]},{cfg['batch_config']['cells']}>",
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "median_launch_ms": statistics.median(per_launch)}

    extras = {}
    e2e = None
    if not args.no_extras and args.workload != "batched":
        e2e = measure_e2e(D, pb, args.precision, dev, stream)
        if args.precision == "fp32" and rank == 0:
            extras["fp64"] = measure_fp64(D, pb, dev, stream)
    if not args.no_extras and args.workload == "kh4096" and args.precision == "fp32" and rank == 0:
        from paper_2006_15932_gb300 import workloads as W

        # a short serving run of a smaller request mix (sides 128..512, 500..2000
        # steps), so that latency percentiles and the sequential-FP64 baseline
        # appear beside the step throughput
        mix = W.serving_requests(48, seed=W.SEED + 2, lo=128, hi=512, steps=(500, 2000))
        extras["serve"] = dict(serve_study(D, dev, mix, 0.8, 128, subset_n=8),
                               mix="48 requests: sides log-uniform 128..512, 2-4 species, half reactive, "
                                   "500..2000 steps, seeded")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "bf16dev": "bf16+f32"}[args.precision],
            "data": "synthetic (seeded analytic initial fields)", "config": cfg, "roofline": roofline,
            "clocks": clk, "gpu_launches": K, "e2e": e2e}
    line.update(extras)
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(pb, args.precision, args.cpu_seconds)
    if args.workload == "batched":
        batch.close()
        for s_ in solvers:
            s_.close()
    else:
        solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measure_e2e(D, pb, precision, dev, stream, n_inner=50, reps=6, lanes=2):
    """End to end through the C ABI with host buffers, as a caller without
    device-side field buffers would use it: every solve hands the library
    page-locked host pointers, so dbm_set_state reads the initial fields
    (rho^s, u_x, u_y, T) straight from host memory, n_inner dbm_step follow,
    and dbm_moments writes the (4S+5) FP64 output fields straight into
    page-locked host memory.  Solves run on `lanes` streams, each with its
    own solver and output buffer, issued in turn, so that one solve's
    host transfers overlap another's steps; the value counts the updates of
    all `reps` solves over the wall time from the first issue to the last
    result on the host.  Bytes per step are each solve's host-to-device and
    device-to-host bytes divided by its n_inner steps."""
    import torch

    host = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
            for a in (pb.rho_s, pb.ux, pb.uy, pb.T)]
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(lanes - 1)]
    lane = []
    for st in streams:
        lane.append({"stream": st, "solver": D.Solver(pb, precision, device=dev, stream=st),
                     "out_host": torch.empty((4 * pb.ns + 5, pb.ny, pb.nx), dtype=torch.float64).pin_memory()})

    def issue(L):
        h, st = L["solver"].h, L["stream"].cuda_stream
        D.dbm_set_state(h, *[t.data_ptr() for t in host], st)
        D.dbm_step(h, n_inner, st)
        D.dbm_moments(h, L["out_host"].data_ptr(), st)

    for L in lane:  # warm-up
        issue(L)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(reps):
        issue(lane[k % lanes])
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t0) / reps
    for L in lane:
        L["solver"].close()
    h2d = sum(h.numel() * 8 for h in host)
    d2h = lane[0]["out_host"].numel() * 8
    return {"value": pb.nx * pb.ny * pb.ns * n_inner / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d / n_inner, "d2h_bytes_per_step": d2h / n_inner,
            "h2d_bytes_per_solve": h2d, "d2h_bytes_per_solve": d2h, "steps_per_solve": n_inner,
            "step": f"one solve: dbm_set_state from page-locked host fields, {n_inner} dbm_step, "
                    f"dbm_moments into page-locked host memory; {reps} solves on {lanes} streams, host wall time"}


def measure_fp64(D, pb, dev, stream, steps=10):
    import torch

    s = D.Solver(pb, "fp64", device=dev, stream=stream)
    with torch.cuda.stream(stream):
        s.set_state()
        s.step(2)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        s.step(steps)
        b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    s.close()
    upd = pb.nx * pb.ny * pb.ns / (ms * 1e-3)
    tflops = upd * FP64_FLOPS_PER_UPDATE / 1e12
    return {"value": upd, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "hbm_frac_of_measured": upd * BYTES_PER_UPDATE["fp64"] / 1e9 / measured_peaks()[0],
            "bound": "alu (FP64 pipe)", "fp64_tflops": tflops, "fp64_frac_of_nominal": tflops / FP64_PEAK_TFLOPS}


if __name__ == "__main__":
    sys.exit(main())
