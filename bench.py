"""Benchmark: MLUPS/species of the fused LBM / Maxwell-Stefan step on GB300.

Default workload: the 3-D D3Q19 ternary anode, 256x128x128 voxels of seeded
overlapping spheres (radius 3, porosity 0.40), inlet H2/H2O/Ar 0.5/0.1/0.4,
1.0 A/cm2, 1073 K, 1 atm, FP32 populations.  A "step" is one time step of
the whole hot path (stream + bounce-back + inlet/outlet + moments + lagged
gradient + Maxwell-Stefan coupling + collision); MLUPS/species counts fluid
cells x 3 species x steps / s.

One JSON line on stdout (rank 0).  ``--impl reference`` times the CPU FP64
oracle instead (a bounded sample of the same workload on the host cores).
Launch with ``torchrun`` for N > 1: every rank runs its own replica (the
method has no cross-replica exchange), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "anode3d_256x128x128": "anode_3d_256x128x128",
    "anode2d_96x48": "anode_2d_96x48",
    "anode3d_512": "anode_3d_512",
    "sweep": None,
    "table2": None,
    "warmstart": None,
}
METRIC = "MLUPS/species"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="anode3d_256x128x128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--time-to-residual", type=float, default=0.0,
                    help="also run to this residual from the uniform start and report the time")
    ap.add_argument("--ttr-forms", default="",
                    help="comma list of time-to-residual forms to run: plain_fp32, plain_fp64, "
                         "fp16_extrapolated, fp32_extrapolated, fp16_extrapolated_profile1d, "
                         "fp16_extrapolated_network (default: plain_fp32 and the three "
                         "extrapolated forms without the network)")
    ap.add_argument("--max-steps", type=int, default=3_000_000)
    ap.add_argument("--step-variant", type=int, default=0,
                    help="0: the autotuner picks the step kernel; k > 0 forces variant k - 1 "
                         "(to profile the variant a plain run picked)")
    ap.add_argument("--extrapolate-every", type=int, default=20000,
                    help="W of the slowest-mode extrapolation in the accelerated time-to-residual run")
    ap.add_argument("--sweep-2d", type=int, default=8, help="2-D microstructures of the sweep")
    ap.add_argument("--sweep-3d", type=int, default=8, help="3-D microstructures of the sweep")
    ap.add_argument("--sweep-scale", type=float, default=1.0, help="size factor of the sweep grids")
    ap.add_argument("--sweep-points", type=int, default=8, help="operating points per microstructure")
    ap.add_argument("--ws-train", type=int, default=128, help="warm start: training anodes")
    ap.add_argument("--ws-test", type=int, default=16, help="warm start: held-out anodes")
    ap.add_argument("--ws-iters", type=int, default=6000, help="warm start: Adam steps")
    ap.add_argument("--ws-lr", type=float, default=1e-3, help="warm start: peak learning rate")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(dist, value, device):
    """The maximum of a per-rank float over every rank of the process group
    (``dist`` None: a single process, the value itself).  Timings are taken
    as the slowest replica's."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_case(name):
    from workloads import cases
    return getattr(cases, WORKLOADS[name])()


def bytes_per_cell(dim, precision):
    """Algorithmic bytes per fluid-cell update (3 species): one read and one
    write of the Q populations of each species and of its mole fraction, at
    the method's precision: populations 8/4/2 bytes, X 8 bytes in FP64 and 4
    in the single-precision forms (160 B per species-update for D3Q19 FP32,
    84 B with 16-bit populations).  The solver's FP32 forms carry X as a
    double-float pair (8 bytes); the second word is its own extra precision,
    not work of the method, and is not counted."""
    q = 9 if dim == 2 else 19
    ps = {"fp64": 8, "fp32": 4, "fp16": 2}[precision]
    xs = 8 if precision == "fp64" else 4
    return 3 * (2 * q * ps + 2 * xs)


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) > 8:
                for k, n in enumerate(names):
                    if r[5 + k].lower() == "active":
                        reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ roofline
def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("lbms_kernels.cuh", "lbms_lattice.cuh", "lbms_launch.cu", "lbms_step_launch.cuh"):
        with open(os.path.join(ROOT, "paper_1809_01600_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def variant_key(info):
    """Step-kernel variant as written in profiles/traffic.txt: cells per block
    x resident blocks, threads per cell, neighbour lookup (32 / 16 bits per
    link, or 1: the per-row fluid bitmasks)."""
    return f"{info.tile_cells}x{info.tile_min_blocks}/t{info.threads_per_cell}/nb{info.neighbour_bits}"


def ncu_traffic(workload, precision, variant):
    """DRAM bytes per launch of the step kernel variant in use, from the
    committed ncu summary; valid only while the kernel sources are unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(p).read().splitlines()
    except OSError:
        return None
    sha = kernel_source_sha()
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        kv = dict(x.split("=", 1) for x in ln.split() if "=" in x)
        if (kv.get("kernel_sha") == sha and kv.get("workload") == workload and kv.get("precision") == precision
                and kv.get("variant") == variant):
            return float(kv["dram_bytes_per_launch"])
    return None


# ------------------------------------------------------------- oracle
def oracle_sample(case, budget_s, steps_hint):
    """A z-slab of the workload (periodic), sized so one oracle step takes
    about budget_s / steps_hint seconds."""
    from oracle import Oracle
    nz = case.solid.shape[0]
    slab = max(1, min(nz, 2))
    probe = case.with_(solid=np.ascontiguousarray(case.solid[:slab]))
    o = Oracle(probe)
    t = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t
    per_plane = per / slab
    target = budget_s / max(1, steps_hint)
    planes = int(max(1, min(nz, target / max(per_plane, 1e-9))))
    return case.with_(solid=np.ascontiguousarray(case.solid[:planes])), planes


def run_oracle(case, steps, warmup):
    from oracle import Oracle
    o = Oracle(case)
    o.step(warmup)
    t = time.perf_counter()
    o.step(steps)
    return time.perf_counter() - t


def cores_used():
    # numpy element-wise kernels run on one thread
    return 1


# ------------------------------------------------------------------ main
def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return main_reference(args, ws, rank)
    if args.workload == "sweep":
        return main_sweep(args, ws, rank, local)
    if args.workload == "table2":
        return main_table2(args, ws, rank, local)
    if args.workload == "warmstart":
        return main_warmstart(args, ws, rank, local)

    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1809_01600_gb300 import lbms as L
    L.load()

    case = make_case(args.workload)
    nf = case.n_fluid
    s = L.Solver.from_case(case, precision=args.precision, step_variant=args.step_variant)
    s.set_bc(case.x_in, case.current_A_cm2)
    stream = torch.cuda.current_stream()
    tinfo = s.info()

    # warm-up: W steps, then one graph-sized batch so the step graph exists
    s.step(args.warmup)
    s.step(32)
    s.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    t_dev = ms / 1e3
    t_dev = max_over_ranks(dist, t_dev, "cuda")
    units = nf * 3 * args.steps * ws
    value = units / t_dev / 1e6

    # dominant kernel = the step kernel, one launch per step
    bpc = bytes_per_cell(case.dim, args.precision)
    per_launch = t_dev / args.steps
    achieved = nf * bpc / per_launch / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = ncu_traffic(case.name, args.precision, variant_key(tinfo))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_kind, "bytes_per_fluid_cell": bpc, "variant": variant_key(tinfo),
                "algorithmic_bytes_per_launch": nf * bpc,
                "kernel": "%s<%s, X %s, h %s>" % (
                    "step_kernel_cell" if tinfo.threads_per_cell == 1 else "step_kernel",
                    "D3Q19" if case.dim == 3 else "D2Q9",
                    "double" if args.precision == "fp64" else "float pair",
                    {"fp64": "double", "fp32": "float", "fp16": "__half"}[args.precision])}

    # time to residual from the uniform start (optional): plain FP32 against
    # the chosen form (FP16 storage + slowest-mode extrapolation)
    ttr = None
    if args.time_to_residual > 0:
        ttr = {"tol": args.time_to_residual}
        forms = (("plain_fp32", "fp32", 0, "uniform"),
                 ("plain_fp64", "fp64", 0, "uniform"),
                 ("fp16_extrapolated", "fp16", args.extrapolate_every, "uniform"),
                 ("fp32_extrapolated", "fp32", args.extrapolate_every, "uniform"),
                 ("fp16_extrapolated_profile1d", "fp16", args.extrapolate_every, "profile1d"),
                 ("fp16_extrapolated_network", "fp16", args.extrapolate_every, "network"))
        pick = (args.ttr_forms.split(",") if args.ttr_forms
                else [f[0] for f in forms if f[0] not in ("plain_fp64", "fp16_extrapolated_network")])
        net = None
        if "fp16_extrapolated_network" in pick:
            from workloads import cases as W_
            net, info = train_warmstart_net(L, W_.warmstart_cases(args.ws_train, 1000), 1e-8, args)
            ttr["network"] = dict(info, note="trained on 64x32x32 anodes; the prediction time is inside "
                                             "the form's seconds, the training is not")
        for label, prec, W, init in forms:
            if label not in pick:
                continue
            r0 = L.Solver.from_case(case, precision=prec, extrapolate_every=W,
                                    init_mode="uniform" if init == "network" else init)
            r0.set_bc(case.x_in, case.current_A_cm2)
            torch.cuda.synchronize()
            t = time.perf_counter()
            if init == "network":
                net.warm_start(r0)
            n, r, st = r0.run_to_residual(args.time_to_residual, args.max_steps, raise_on_fail=False)
            ttr_s = time.perf_counter() - t
            eta, _ = r0.overpotential()
            ttr[label] = {"precision": prec, "extrapolate_every": W, "init": init, "steps": n, "residual": r,
                          "seconds": round(ttr_s, 3), "converged": st == L.LBMS_OK, "eta_V": eta}
            r0.close()
        if net is not None:
            net.close()
        base = ttr.get("plain_fp32")
        for label, _, _, _ in forms[1:]:
            if base and label in ttr:
                ttr[label]["speedup_vs_plain_fp32"] = round(base["seconds"] / ttr[label]["seconds"], 2)
                ttr[label]["eta_rel_diff_vs_plain_fp32"] = abs(ttr[label]["eta_V"] - base["eta_V"]) / abs(base["eta_V"])

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t = time.perf_counter()
        s2 = L.Solver.from_case(case, precision=args.precision, step_variant=args.step_variant)
        s2.set_bc(case.x_in, case.current_A_cm2)
        s2.step(args.steps)
        X = s2.fields()
        eta, _ = s2.overpotential()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t
        info = s2.info()
        s2.close()
        t_e2e = max_over_ranks(dist, t_e2e, "cuda")
        e2e = {"value": round(units / t_e2e / 1e6, 2), "unit": METRIC,
               "h2d_bytes_per_step": int(info.h2d_bytes / args.steps),
               "d2h_bytes_per_step": int(info.d2h_bytes / args.steps),
               "seconds": round(t_e2e, 3),
               "scope": "create from host mask + set_bc + K steps + fields to host + overpotential"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample, planes = oracle_sample(case, 20.0, 2)
        t_cpu = run_oracle(sample, 2, 0)
        cpu = {"value": round(sample.n_fluid * 3 * 2 / t_cpu / 1e6, 4), "unit": METRIC,
               "cores": cores_used(), "kind": "oracle",
               "sample": f"2 FP64 oracle steps on the first {planes} z-planes of the same "
                         f"{case.name} mask ({sample.n_fluid} fluid cells, periodic in z)"}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": METRIC, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f32 (f16 storage)"}[args.precision],
                "data": "synthetic",
                "config": {"workload": case.name, "lattice": "D3Q19" if case.dim == 3 else "D2Q9",
                           "grid": list(case.solid.shape[::-1]), "fluid_cells": nf,
                           "porosity": round(case.porosity, 4), "current_A_cm2": case.current_A_cm2,
                           "x_in": list(case.x_in), "precision": args.precision,
                           "parallelism": f"replicas x{ws}",
                           "tile": f"{tinfo.tile_cells} cells per block, "
                                   f"{'one thread per cell' if tinfo.threads_per_cell == 1 else 'one thread per cell and species'}, "
                                   f"{tinfo.tile_min_blocks} blocks/SM, {tinfo.neighbour_bits}-bit "
                                   f"neighbour table (autotuned)",
                           "l2": "state larger than L2 (no flush needed)" if nf * bpc > 129e6 * 2
                           else "state fits in L2"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": args.steps, "time_to_residual": ttr}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def sweep_cases(args):
    """The uneven-size sweep: each microstructure at each operating point."""
    from workloads import cases as W
    structs = W.sweep_structures(args.sweep_2d, args.sweep_3d, scale=args.sweep_scale)
    pts = W.sweep_operating_points(args.sweep_points)
    groups = {2: [], 3: []}
    for st in structs:
        for I, x in pts:
            groups[st.dim].append(st.with_(current_A_cm2=I, x_in=x))
    return groups


def train_warmstart_net(L, train, tol, args):
    """Steady states of the training anodes (one batch, FP32 + extrapolation)
    and a warm-start network trained on them; returns the net and timings."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = L.Batch.from_cases(train, precision="fp32", extrapolate_every=5000)
    for k, c in enumerate(train):
        b.set_bc(c.x_in, c.current_A_cm2, case=k)
    n, _, _, st = b.run_to_residual(tol, args.max_steps, raise_on_fail=False)
    net = L.Net(width=704, depth=3, seed=1)
    for k in range(len(train)):
        net.add_sample(b, k)
    b.close()
    t1 = time.perf_counter()
    loss = net.train(args.ws_iters, batch=8192, lr=args.ws_lr)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, {"data": {"cases": len(train), "rows": net.info()[1], "steps": int(n),
                          "seconds": round(t1 - t0, 2)},
                 "training": {"params": net.info()[0], "iters": args.ws_iters, "batch": 8192, "lr": args.ws_lr,
                              "final_loss": loss, "seconds": round(t2 - t1, 2)}}


def main_warmstart(args, ws, rank, local):
    """Learned warm start: steady states of seeded 64x32x32 anodes from the
    batched solver train the network; on held-out anodes, the steps to
    residual 1e-8 from the uniform start, the 1-D profile of Section 4.1 and
    the network's prediction (plain FP32, and FP16 storage + extrapolation)."""
    import torch
    torch.cuda.set_device(local)
    from paper_1809_01600_gb300 import lbms as L
    from workloads import cases as W
    L.load()
    tol = args.time_to_residual or 1e-8
    train = W.warmstart_cases(args.ws_train, 1000)
    test = W.warmstart_cases(args.ws_test, 5000)
    out = {"residual": tol}

    net, info = train_warmstart_net(L, train, tol, args)
    out.update(info)

    forms = (("plain_fp32", "fp32", 0), ("fp16_extrapolated", "fp16", 5000))
    for label, prec, Wx in forms:
        res = {}
        for start in ("uniform", "profile1d", "network"):
            bt = L.Batch.from_cases(test, precision=prec, extrapolate_every=Wx,
                                    init_mode="profile1d" if start == "profile1d" else "uniform")
            for k, c in enumerate(test):
                bt.set_bc(c.x_in, c.current_A_cm2, case=k)
            torch.cuda.synchronize()
            ta = time.perf_counter()
            if start == "network":
                for k in range(len(test)):
                    net.warm_start(bt, k)
            torch.cuda.synchronize()
            tb = time.perf_counter()
            n, steps, r, st = bt.run_to_residual(tol, args.max_steps, raise_on_fail=False)
            torch.cuda.synchronize()
            tc = time.perf_counter()
            res[start] = {"mean_steps": float(np.mean(steps)), "max_steps": int(np.max(steps)),
                          "converged": bool(np.all(steps > 0)), "start_seconds": round(tb - ta, 3),
                          "batch_seconds": round(tc - tb, 2)}
            bt.close()
        for start in ("profile1d", "network"):
            res[start]["steps_vs_uniform"] = round(res[start]["mean_steps"] / res["uniform"]["mean_steps"], 3)
        out[label] = res
    net.close()
    if rank == 0:
        v = out["plain_fp32"]["network"]["mean_steps"]
        line = {"metric": "steps to residual (held-out anodes, network start)", "value": v, "unit": "steps",
                "n_gpus": 1, "higher_is_better": False, "vs_baseline": None, "dtype": "bf16 network, f32 LBM",
                "data": "synthetic",
                "config": {"workload": f"learned warm start, {len(train)} training + {len(test)} held-out "
                                       f"64x32x32 D3Q19 anodes"},
                "warm_start": out}
        print(json.dumps(line))
    return 0


def main_table2(args, ws, rank, local):
    """The homogenised anode of Section 4.2 (Table 2 gas point): every current
    of Figs. 2-4 x every inlet dilution in one batch, run to steady state
    (residual 1e-8, or --time-to-residual) from the uniform inlet start;
    reports the steady eta - eta_0 table and the time to get it."""
    import torch
    torch.cuda.set_device(local)
    from paper_1809_01600_gb300 import lbms as L
    from workloads import cases as W
    L.load()
    tol = args.time_to_residual or 1e-8
    cs = W.paper_table2_cases(64)
    b = L.Batch.from_cases(cs, precision=args.precision)
    for k, c in enumerate(cs):
        b.set_bc(c.x_in, c.current_A_cm2, case=k)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    n, steps, r, status = b.run_to_residual(tol, args.max_steps, raise_on_fail=False)
    eta, _ = b.overpotentials(raise_on_fail=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    b.close()
    nh = len(W.TABLE2_H2)
    e = np.asarray(eta).reshape(len(W.TABLE2_CURRENTS), nh)
    table = {f"{I} A/cm2": {f"xH2={xh}": round(float(e[i, j] - e[i, 0]), 6)
                            for j, xh in enumerate(W.TABLE2_H2) if j > 0}
             for i, I in enumerate(W.TABLE2_CURRENTS)}
    nf = sum(c.n_fluid for c in cs)
    if rank == 0:
        line = {"metric": "time to residual", "value": round(wall, 3), "unit": "s", "n_gpus": 1,
                "higher_is_better": False, "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f32 (f16 storage)"}[args.precision],
                "data": "synthetic",
                "config": {"workload": "homogenised Table 2 anode, 1-D D2Q9 strip nx=64, "
                                       f"{len(W.TABLE2_CURRENTS)} currents x {nh} inlets in one batch",
                           "residual": tol, "fluid_cells": nf, "precision": args.precision},
                "steps": int(n), "steps_per_case": [int(x) for x in steps],
                "converged": bool(np.all(steps > 0)), "status": int(status),
                "eta_V_minus_eta0_V": table, "clocks": clk}
        print(json.dumps(line))
    return 0


def main_sweep(args, ws, rank, local):
    """Many microstructures x operating points: one launch per lattice and
    step (batched, autotuned tile) against stepping every case in a handle
    of its own."""
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1809_01600_gb300 import lbms as L
    L.load()
    groups = sweep_cases(args)
    batches = []
    for dim in (2, 3):
        cs = groups[dim]
        if not cs:
            continue
        b = L.Batch.from_cases(cs, precision=args.precision)
        for k, c in enumerate(cs):
            b.set_bc(c.x_in, c.current_A_cm2, case=k)
        batches.append((dim, cs, b))
    nf = sum(c.n_fluid for _, cs, _ in batches for c in cs)
    stream = torch.cuda.current_stream()
    for _, _, b in batches:
        b.step(args.warmup)
        b.step(32)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _, _, b in batches:
        b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    t_dev = ms / 1e3
    t_dev = max_over_ranks(dist, t_dev, "cuda")
    units = nf * 3 * args.steps * ws
    value = units / t_dev / 1e6
    tiles = {dim: "%d cells, %d blocks/SM" % (b.info().tile_cells, b.info().tile_min_blocks)
             for dim, _, b in batches}
    etas = {dim: b.overpotentials(raise_on_fail=False)[0] for dim, _, b in batches}
    for _, _, b in batches:
        b.close()

    # the same cases, one handle each, stepped one after another
    seq_steps = max(1, min(args.steps, 200))
    t_seq = 0.0
    for dim in (2, 3):
        for c in groups[dim]:
            s = L.Solver.from_case(c, precision=args.precision)
            s.set_bc(c.x_in, c.current_A_cm2)
            s.step(32)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            s.step(seq_steps)
            a1.record(stream)
            torch.cuda.synchronize()
            t_seq += a0.elapsed_time(a1) / 1e3
            s.close()
    seq_value = nf * 3 * seq_steps / t_seq / 1e6
    bpc = {d: bytes_per_cell(d, args.precision) for d in (2, 3)}
    alg = sum(c.n_fluid * bpc[c.dim] for _, cs, _ in batches for c in cs)
    achieved = alg / (t_dev / args.steps) / 1e9
    peak, peak_kind = measured_peak_hbm()
    if rank == 0:
        n2, n3 = len(groups[2]), len(groups[3])
        line = {"metric": METRIC, "value": round(value, 2), "unit": METRIC, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f32 (f16 storage)"}[args.precision],
                "data": "synthetic",
                "config": {"workload": f"sweep of {args.sweep_2d} 2-D + {args.sweep_3d} 3-D microstructures "
                                       f"x {args.sweep_points} operating points",
                           "cases": {"2d": n2, "3d": n3}, "fluid_cells": nf, "precision": args.precision,
                           "tiles": tiles, "parallelism": f"replicas x{ws}",
                           "launches_per_step": len(batches)},
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_kind},
                "sequential": {"value": round(seq_value, 2), "unit": METRIC,
                               "what": "the same cases, one handle each, stepped one after another",
                               "steps": seq_steps},
                "speedup_vs_sequential": round(value / seq_value, 2),
                "eta_V_range": [float(np.nanmin(np.concatenate(list(etas.values())))),
                                float(np.nanmax(np.concatenate(list(etas.values()))))],
                "clocks": clk, "gpu_launches": args.steps * len(batches)}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main_reference(args, ws, rank):
    if rank != 0:
        return 0
    case = make_case(args.workload)
    budget = 150.0
    sample, planes = oracle_sample(case, budget, args.steps + args.warmup)
    t = run_oracle(sample, args.steps, args.warmup)
    value = sample.n_fluid * 3 * args.steps / t / 1e6
    desc = (f"FP64 CPU oracle on the first {planes} z-planes of the {case.name} mask "
            f"({sample.n_fluid} fluid cells, periodic in z), {args.steps} timed steps")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": METRIC,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case.name, "precision": args.precision,
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": round(value, 4), "unit": METRIC, "cores": cores_used(),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 4), "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
