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
                                                                    "precision_kh", "precision_reactive"])
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


def make_workload(name, grid=None):
    from paper_2006_15932_gb300 import workloads as W

    nx, ny = (int(v) for v in grid.lower().split("x")) if grid else (None, None)
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
                     "serve": "serve_poisson_request_mix"}[name],
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


def cpu_baseline(pb_full, precision, seconds):
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
    O.run(p, f, 1)  # start the OpenMP thread pool
    t0 = time.perf_counter()
    f, st = O.run(p, f, 1)
    t1 = time.perf_counter()
    per_step = max(t1 - t0, 1e-6)
    steps = max(1, min(1000, int(seconds / per_step)))
    t0 = time.perf_counter()
    _, st2 = O.run(p, f, steps)
    dt = time.perf_counter() - t0
    if st or st2:
        raise RuntimeError(f"oracle status {st}/{st2} on the CPU-baseline sample: the timing would be cut short")
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": nx * ny * pb.ns * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nx}x{ny} window of the {pb_full.nx}x{pb_full.ny} grid, {pb.ns} species, "
                      f"{steps} FP64 steps in {dt:.1f} s (OpenMP over rows)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pb = make_workload(args.workload, args.grid)
    cfg = workload_config(pb, args.workload, args.precision)
    # each "step" of the reference arm is a bounded sample of the workload
    per = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(pb, args.precision, per / 4)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(pb, args.precision, per))
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


def run_serve(args, D, dev):
    """Serving: Poisson arrivals of the request mix at a fraction of the
    measured capacity, continuous batching; p50/p99 latency and throughput,
    against first-come-first-served sequential solves (FP64 and unbatched
    FP32) whose service times come from throughputs measured here."""
    import torch

    from paper_2006_15932_gb300 import serve as SV
    from paper_2006_15932_gb300 import workloads as W

    s_lo, s_hi = (int(v) for v in args.serve_sides.split(","))
    n_lo, n_hi = (int(v) for v in args.serve_steps.split(","))
    specs = W.serving_requests(args.serve_requests, lo=s_lo, hi=s_hi, steps=(n_lo, n_hi))
    # capacity: the same mix (other seed, 1/20 of the steps) all arriving at once
    cal = W.serving_requests(32, seed=W.SEED + 1, lo=s_lo, hi=s_hi,
                             steps=(max(1, n_lo // 20), max(2, n_hi // 20)))
    SV.Server(device=dev, qmax=args.serve_qmax).run(cal[:4])  # warm-up: kernels, allocator
    cap = SV.summarize(SV.Server(device=dev, qmax=args.serve_qmax).run(cal))["throughput"]
    mean_units = sum(s.units for s in specs) / len(specs)
    rate = args.serve_load * cap / mean_units
    specs = W.poisson_arrivals(specs, rate)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    srv = SV.Server(device=dev, qmax=args.serve_qmax)
    res = srv.run(specs)
    clk = clocks.stop()
    if any(r.status for r in res):
        raise SystemExit("health flag raised while serving")
    summ = SV.summarize(res)

    # sequential references: FP64 and unbatched FP32 throughput per species
    # count on a 512 x 512 shock tube (FP64 is ALU-bound, so its rate hardly
    # depends on the size)
    def rate_of(precision, ns, steps):
        spec = W.RequestSpec(rid=0, kind="shock", L=512, ns=ns, seed=1, nsteps=steps)
        st = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(st):
            s = D.Solver(W.request_problem(spec), precision, device=dev)
            s.set_state(*W.request_fields(spec, dev))
            s.step(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.step(steps)
            e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        return 512 * 512 * ns * steps / (ms * 1e-3)

    nss = sorted({s.ns for s in specs})
    r64 = {ns: rate_of("fp64", ns, 4) for ns in nss}
    r32 = {ns: rate_of("fp32", ns, 200) for ns in nss}
    seq64 = SV.simulate_sequential(specs, r64)
    seq32 = SV.simulate_sequential(specs, r32)
    peak, peak_kind = measured_peaks()
    bpu = BYTES_PER_UPDATE["fp32"]
    cfg = {"workload": "serve_poisson_request_mix", "requests": len(specs), "sides": [s_lo, s_hi],
           "side_distribution": "log-uniform", "species": nss, "reactive_fraction": 0.5,
           "steps": [n_lo, n_hi], "precision": "fp32", "arrival_rate_per_s": rate,
           "load": args.serve_load, "capacity_units_per_s": cap, "qmax": args.serve_qmax,
           "batch_config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in srv.config.items()},
           "l2_policy": "inputs larger than L2"}
    line = {"metric": METRIC, "value": summ["throughput"], "unit": UNIT, "n_gpus": 1, "steps": len(specs),
            "warmup": 4, "ms_per_step": 1e3 * summ["makespan_s"] / len(specs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded request mix, Poisson arrivals)", "config": cfg,
            "serve": {"p50_s": summ["p50_s"], "p99_s": summ["p99_s"], "mean_s": summ["mean_s"],
                      "makespan_s": summ["makespan_s"], "units": summ["units"],
                      "hbm_budget_bytes": srv.adm.budget, "admitted_peak_bytes": srv.adm.peak,
                      "batch_rebuilds": sum(g.rebuilds for g in srv.groups.values()),
                      "quanta": srv.launch_quanta,
                      "hbm_frac_whole_run": summ["throughput"] * bpu / 1e9 / peak},
            "fp64_sequential": dict(seq64, rate_by_species=r64,
                                    how="FIFO one request at a time; service = units / FP64 rate measured "
                                        "on a 512x512 tube per species count"),
            "fp32_unbatched_sequential": dict(seq32, rate_by_species=r32,
                                              how="FIFO one request at a time; service = units / single-"
                                                  "problem FP32 rate measured on a 512x512 tube"),
            "clocks": clk, "e2e": {"value": summ["throughput"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                   "d2h_bytes_per_step": 8 * (max(nss) + 4)},
            "roofline": {"bound": "hbm", "achieved": summ["throughput"] * bpu / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": summ["throughput"] * bpu / 1e9 / peak, "traffic": None,
                         "kernel": "all step kernels of the run (whole-run average)",
                         "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args, D, dev):
    """Precision study: the same initial state advanced in FP64, FP32 and
    BF16DEV (the latter only where its scope allows), relative L2 and
    L-infinity errors of the mixture fields against FP64 at checkpoints, and
    each precision's drift of the conserved totals over the run."""
    import torch

    from paper_2006_15932_gb300 import workloads as W

    if args.workload == "precision_kh":
        nx, ny = (int(v) for v in (args.grid or "4096x4096").lower().split("x"))
        pb = W.kh_shear_layer(nx, ny=ny)
        total = args.study_steps or 1000
        precs = ["fp64", "fp32", "bf16dev"]
        checkpoints = 4
    else:
        nx, ny = (int(v) for v in (args.grid or "1024x256").lower().split("x"))
        pb = W.reactive_premixed(nx, ny)
        total = args.study_steps or 20000
        precs = ["fp64", "fp32"]
        checkpoints = 10
    st = torch.cuda.Stream(device=dev)
    sols = {}
    with torch.cuda.stream(st):
        for p in precs:
            sols[p] = D.Solver(pb, p, device=dev)
            sols[p].set_state()
        cons0 = {p: sols[p].conservation().cpu().numpy() for p in precs}
    S = pb.ns
    names = ["rho", "ux", "uy", "T"]
    rows = {"rho": 4 * S, "ux": 4 * S + 1, "uy": 4 * S + 2, "T": 4 * S + 3}
    # velocity errors are measured against the velocity scale of the run
    # (max |u| of the FP64 field, at least the sound speed 1), not against a
    # field that may vanish
    curve = []
    per = total // checkpoints
    done = 0
    t_fp64 = 0.0
    while done < total:
        n = min(per, total - done)
        with torch.cuda.stream(st):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sols["fp64"].step(n)
            e1.record(st)
            for p in precs[1:]:
                sols[p].step(n)
            mom = {p: sols[p].moments() for p in precs}
        st.synchronize()
        t_fp64 += e0.elapsed_time(e1) * 1e-3
        done += n
        ref = mom["fp64"]
        entry = {"step": done}
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
    drift = {}
    with torch.cuda.stream(st):
        for p in precs:
            c1 = sols[p].conservation().cpu().numpy()
            c0 = cons0[p]
            mass0 = float(sum(abs(c0[:S])))
            e_scale = abs(float(c0[S + 2])) + abs(float(c0[S + 3]))
            drift[p] = {"mass": float(abs(sum(c1[:S]) - sum(c0[:S])) / mass0),
                        "momentum_x": float(abs(c1[S] - c0[S]) / mass0),
                        "momentum_y": float(abs(c1[S + 1] - c0[S + 1]) / mass0),
                        "energy_plus_bound_heat": float(abs((c1[S + 2] + c1[S + 3]) - (c0[S + 2] + c0[S + 3]))
                                                        / e_scale)}
    for p in precs:
        rc, bits = sols[p].status()
        if rc != 0:
            raise SystemExit(f"health flag raised in {p}: bits={bits}")
        sols[p].close()
    line = {"study": args.workload, "grid": [pb.nx, pb.ny], "species": S, "steps": total,
            "boundary": ["periodic" if b == 0 else "outflow" for b in (pb.bc_x, pb.bc_y)],
            "reactive": pb.k_ov != 0.0, "fp64_seconds": t_fp64,
            "error_vs_fp64": curve, "conservation_drift": drift,
            "norms": "rel_linf = max|a-b| / max|b|, rel_l2 = ||a-b|| / ||b||; for u_x, u_y the scale is "
                     "max(max|u|, 1) (and rms of that scale for L2)"}
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
        pb = make_workload(args.workload, args.grid)
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
                else f"k_step_batch<{pb.ns},{cfg['tile'][0]},{cfg['tile'][1]}>",
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "median_launch_ms": statistics.median(per_launch)}

    extras = {}
    e2e = None
    if not args.no_extras and args.workload != "batched":
        e2e = measure_e2e(D, pb, args.precision, dev, stream)
        if args.precision == "fp32" and rank == 0:
            extras["fp64"] = measure_fp64(D, pb, dev, stream)
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
    """End to end through the public API: pinned host fields -> device,
    dbm_set_state, n_inner dbm_step, dbm_moments, moments -> pinned host.
    Every solve copies its inputs in and its result out.  Solves run on
    `lanes` streams, each with its own solver and buffers, issued in turn,
    so that one solve's copies overlap another's kernels, as a caller
    serving a stream of solves would run them; the value counts the updates
    of all `reps` solves over the wall time from the first issue to the last
    result on the host."""
    import torch

    host = [torch.from_numpy(a.astype("float64")).pin_memory() for a in (pb.rho_s, pb.ux, pb.uy, pb.T)]
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(lanes - 1)]
    lane = []
    for st in streams:
        with torch.cuda.stream(st):
            lane.append({"stream": st, "solver": D.Solver(pb, precision, device=dev),
                         "dev_in": [torch.empty(h.shape, dtype=torch.float64, device=dev) for h in host],
                         "dev_out": torch.empty((4 * pb.ns + 5, pb.ny, pb.nx), dtype=torch.float64, device=dev),
                         "out_host": torch.empty((4 * pb.ns + 5, pb.ny, pb.nx), dtype=torch.float64).pin_memory()})

    def issue(L):
        with torch.cuda.stream(L["stream"]):
            for d, h in zip(L["dev_in"], host):
                d.copy_(h, non_blocking=True)
            L["solver"].set_state(*L["dev_in"])
            L["solver"].step(n_inner)
            L["solver"].moments(L["dev_out"])
            L["out_host"].copy_(L["dev_out"], non_blocking=True)

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
    return {"value": pb.nx * pb.ny * pb.ns * n_inner / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "step": f"one solve: host fields in, dbm_set_state, {n_inner} dbm_step, dbm_moments, host out; "
                    f"{reps} solves on {lanes} streams, host wall time"}


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
