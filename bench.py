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
    "anode3d_small": "anode_3d_small",
    "sweep": None,
    "table2": None,
    "warmstart": None,
    "unet": None,
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
    ap.add_argument("--no-fp16-line", action="store_true",
                    help="skip the throughput of the 16-bit storage form in the FP32 line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--time-to-residual", type=float, default=1e-8,
                    help="run each time-to-residual form to this residual and report the time "
                         "(the second half of the metric); 0 or --no-ttr skips it")
    ap.add_argument("--no-ttr", action="store_true", help="skip the time-to-residual forms")
    ap.add_argument("--ttr-forms", default="plain_fp32,fp16_extrapolated_network",
                    help="comma list of time-to-residual forms: plain_fp32, plain_fp64, "
                         "fp16_extrapolated, fp32_extrapolated, fp16_extrapolated_profile1d, "
                         "fp16_extrapolated_network (the chosen form: network start, FP16 "
                         "storage, extrapolation)")
    ap.add_argument("--no-ttr-reference", action="store_true",
                    help="skip the overpotential reference (FP32 run on to its floor, FP64 polish)")
    ap.add_argument("--ref-tol", type=float, default=3e-10,
                    help="residual the FP32 leg of the overpotential reference runs to")
    ap.add_argument("--ref-fp64-steps", type=int, default=20000,
                    help="FP64 steps that polish the overpotential reference")
    ap.add_argument("--oracle-procs", type=int, default=0,
                    help="oracle processes for the CPU baseline (0: one per host core)")
    ap.add_argument("--oracle-ttr", action="store_true",
                    help="--impl reference: also run the oracle to the residual on the workload")
    ap.add_argument("--max-steps", type=int, default=3_000_000)
    ap.add_argument("--step-variant", type=int, default=0,
                    help="0: the autotuner picks the step kernel; k > 0 forces variant k - 1 "
                         "(to profile the variant a plain run picked)")
    ap.add_argument("--extrapolate-every", type=int, default=20000,
                    help="W of the slowest-mode extrapolation in the accelerated time-to-residual run")
    ap.add_argument("--rre-every", type=int, default=10000,
                    help="W of the reduced-rank extrapolation forms (snapshots W steps apart)")
    ap.add_argument("--rre-modes", type=int, default=4,
                    help="order M of the reduced-rank extrapolation forms (M + 1 snapshots)")
    ap.add_argument("--ttr-chosen", default="fp16_extrapolated_network",
                    help="the form reported as the chosen one (its end state seeds the reference)")
    ap.add_argument("--sweep-2d", type=int, default=32, help="2-D microstructures of the sweep")
    ap.add_argument("--sweep-3d", type=int, default=32, help="3-D microstructures of the sweep")
    ap.add_argument("--sweep-scale", type=float, default=1.0, help="size factor of the sweep grids")
    ap.add_argument("--sweep-points", type=int, default=8, help="operating points per microstructure")
    ap.add_argument("--sweep-small-scale", type=float, default=0.25,
                    help="size factor of the small-case sweep timed batched against one handle per case "
                         "(0 skips it)")
    ap.add_argument("--ws-train", type=int, default=128, help="warm start: training anodes")
    ap.add_argument("--ws-test", type=int, default=16, help="warm start: held-out anodes")
    ap.add_argument("--ws-iters", type=int, default=6000, help="warm start: Adam steps")
    ap.add_argument("--ws-lr", type=float, default=1e-3, help="warm start: peak learning rate")
    ap.add_argument("--ws-test-shape", default="64x32x32",
                    help="warm start: grid (nx x ny x nz) of the held-out anodes")
    ap.add_argument("--ws-train-test-shape", type=int, default=0,
                    help="warm start: training anodes at the held-out grid, added to the 64x32x32 ones")
    ap.add_argument("--ws-plain", action="store_true",
                    help="warm start: also time plain FP32 (no extrapolation) from each start")
    ap.add_argument("--ws-compare-unet", action="store_true",
                    help="warm start: also train the same 3-D U-Net with PyTorch convolutions (a comparison "
                         "arm for the U-Net on this project's kernels) on the same data and time its starts")
    ap.add_argument("--ws-unet-iters", type=int, default=6000,
                    help="warm start: Adam steps of the 3-D U-Net on this project's kernels (0 skips it)")
    ap.add_argument("--ws-unet-width", type=int, default=28, help="warm start: U-Net width (28: 1.05M parameters)")
    ap.add_argument("--ws-starts", default="uniform,profile1d,network,unet",
                    help="warm start: the starts timed on the held-out anodes")
    ap.add_argument("--unet-shape", default="96x96x96", help="--workload unet: volume grid (nx x ny x nz)")
    ap.add_argument("--unet-batch", type=int, default=8, help="--workload unet: volumes per training step")
    ap.add_argument("--unet-steps", type=int, default=20, help="--workload unet: timed training steps")
    ap.add_argument("--unet-torch", action="store_true",
                    help="--workload unet: also time the same U-Net with PyTorch convolutions (TF32 and BF16 "
                         "autocast) on the same volumes")
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
def run_oracle(case, steps, warmup):
    from oracle import Oracle
    o = Oracle(case)
    o.step(warmup)
    t = time.perf_counter()
    o.step(steps)
    return time.perf_counter() - t


def _oracle_slab(workload, z0, z1, steps, warmup, barrier, queue):
    """One oracle process: z-planes [z0, z1) of the workload's mask (periodic
    in z), `warmup` untimed steps, then `steps` timed ones between wall-clock
    stamps taken after every process has warmed up."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import Oracle
    case = make_case(workload)
    sub = case.with_(solid=np.ascontiguousarray(case.solid[z0:z1]))
    o = Oracle(sub)
    o.step(warmup)
    barrier.wait()
    t0 = time.time()
    o.step(steps)
    queue.put((sub.n_fluid, t0, time.time()))


def oracle_all_cores(workload, steps, warmup, procs=0, planes=0):
    """The FP64 oracle on every host core: the first `planes` z-planes of the
    workload (0: all) split into one slab per process (each slab periodic in
    z), run concurrently; returns (fluid cells, wall seconds of the timed
    steps, processes, planes)."""
    import multiprocessing as mp
    case = make_case(workload)
    nz = planes or case.solid.shape[0]
    procs = max(1, min(procs or os.cpu_count() or 1, nz))
    bounds = [(k * nz // procs, (k + 1) * nz // procs) for k in range(procs)]
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    queue = ctx.Queue()
    ps = [ctx.Process(target=_oracle_slab, args=(workload, z0, z1, steps, warmup, barrier, queue))
          for z0, z1 in bounds]
    for p in ps:
        p.start()
    res = [queue.get() for _ in ps]
    for p in ps:
        p.join()
    cells = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return cells, wall, procs, nz


def cores_used():
    # numpy element-wise kernels run on one thread per process
    return 1


# ------------------------------------------------------- throughput / ttr
def time_steps(L, case, precision, args, dist):
    """Throughput of one more handle of the workload at `precision`: the
    same warm-up and CUDA-event timing as the main line, with its roofline
    on the algorithmic bytes of that precision."""
    import torch
    s = L.Solver.from_case(case, precision=precision)
    s.set_bc(case.x_in, case.current_A_cm2)
    info = s.info()
    s.step(args.warmup)
    s.step(32)
    s.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    s.close()
    t_dev = max_over_ranks(dist, ms / 1e3, "cuda")
    nf = case.n_fluid
    bpc = bytes_per_cell(case.dim, precision)
    achieved = nf * bpc / (t_dev / args.steps) / 1e9
    peak, peak_kind = measured_peak_hbm()
    return {"precision": precision, "ms_per_step": round(ms / args.steps, 5),
            "value": round(nf * 3 * args.steps * (dist.get_world_size() if dist else 1) / t_dev / 1e6, 2),
            "unit": METRIC, "clocks": clk,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                         "bytes_per_fluid_cell": bpc, "variant": variant_key(info),
                         "traffic": ncu_traffic(case.name, precision, variant_key(info))}}


def _run_form(L, case, label, prec, W, init, tol, args, net=None, X0=None, modes=1, unet=None):
    """One time-to-residual run on a fresh handle, timed from its boundary
    data being set (the network's prediction, when it starts from one, is
    inside the time) to the residual check that meets tol; clocks sampled
    over the run."""
    import torch
    s = L.Solver.from_case(case, precision=prec, extrapolate_every=W, extrapolate_modes=modes,
                           init_mode="profile1d" if init == "profile1d" else "uniform")
    s.set_bc(case.x_in, case.current_A_cm2)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t = time.perf_counter()
    if init == "network":
        net.warm_start(s)
    elif init == "unet":
        unet.warm_start(s)
    elif X0 is not None:
        s.set_fields(X0)
    n, r, st = s.run_to_residual(tol, args.max_steps, raise_on_fail=False)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t
    clk = clocks.stop()
    eta, xo = s.overpotential()
    info = s.info()
    out = {"precision": prec, "extrapolate_every": W, "extrapolate_modes": modes, "init": init,
           "steps": int(n), "residual": r,
           "seconds": round(secs, 3), "converged": st == L.LBMS_OK, "eta_V": eta,
           "variant": variant_key(info), "clocks": clk}
    return s, out


def time_to_residual(L, case, args):
    """Time to residual tol from the start of each form, plain FP32 against
    the chosen form (network start + FP16 storage + extrapolation), and the
    overpotential of each against a reference steady state: the chosen
    form's end state run on in FP32 with extrapolation to its floor
    (residual --ref-tol), then --ref-fp64-steps FP64 steps."""
    tol = args.time_to_residual
    Wx, Wr, M = args.extrapolate_every, args.rre_every, args.rre_modes
    forms = {"plain_fp32": ("fp32", 0, "uniform", 1),
             "plain_fp64": ("fp64", 0, "uniform", 1),
             "fp16_extrapolated": ("fp16", Wx, "uniform", 1),
             "fp32_extrapolated": ("fp32", Wx, "uniform", 1),
             "fp16_extrapolated_profile1d": ("fp16", Wx, "profile1d", 1),
             "fp16_extrapolated_network": ("fp16", Wx, "network", 1),
             "fp16_extrapolated_unet": ("fp16", Wx, "unet", 1),
             "fp32_rre": ("fp32", Wr, "uniform", M),
             "fp16_rre": ("fp16", Wr, "uniform", M),
             "fp16_rre_network": ("fp16", Wr, "network", M)}
    pick = [f for f in args.ttr_forms.split(",") if f]
    for f in pick:
        if f not in forms:
            raise SystemExit(f"unknown time-to-residual form {f}")
    chosen = args.ttr_chosen if args.ttr_chosen in pick else pick[-1]
    out = {"tol": tol, "chosen": chosen, "baseline": "plain_fp32"}
    net = unet = None
    if any(forms[f][2] in ("network", "unet") for f in pick):
        import torch
        from workloads import cases as W_
        if any(forms[f][2] == "unet" for f in pick):
            vox = int(np.prod([(d + 3) // 4 * 4 for d in case.solid.shape]))
            unet = L.UNet(width=args.ws_unet_width, max_voxels=max(8 * 64 * 32 * 32, vox), seed=1)
        net, info = train_warmstart_net(L, W_.warmstart_cases(args.ws_train, 1000), 1e-8, args, unet=unet)
        out["network"] = dict(info, note="trained on 64x32x32 anodes, none of them this one; the "
                                         "training is outside the form's seconds, the prediction inside")
        if unet is not None:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            uloss = unet.train(args.ws_unet_iters, max_batch=8, lr=args.ws_lr)
            torch.cuda.synchronize()
            out["unet"] = {"params": unet.info()[0], "iters": args.ws_unet_iters, "final_loss": uloss,
                           "seconds": round(time.perf_counter() - t0, 2),
                           "note": "the same 64x32x32 steady states; training outside the form's seconds"}
    start = None      # end state of the chosen form: where the reference starts
    for label in pick:
        prec, W, init, modes = forms[label]
        s, res = _run_form(L, case, label, prec, W, init, tol, args, net=net, modes=modes, unet=unet)
        out[label] = res
        if label == chosen:
            start = s.fields()
        s.close()
    if net is not None:
        net.close()
    if unet is not None:
        unet.close()
    base = out.get("plain_fp32")
    for label in pick:
        if base and label != "plain_fp32":
            out[label]["speedup_vs_plain_fp32"] = round(base["seconds"] / out[label]["seconds"], 2)
    # overpotential reference: continue from the last form's state
    if not args.no_ttr_reference and start is not None:
        ref32, r32 = _run_form(L, case, "reference_fp32", "fp32", Wr, "uniform", args.ref_tol, args,
                               X0=start, modes=M)
        X = ref32.fields()
        ref32.close()
        import torch
        s64 = L.Solver.from_case(case, precision="fp64")
        s64.set_bc(case.x_in, case.current_A_cm2)
        s64.set_fields(X)
        t = time.perf_counter()
        s64.step(args.ref_fp64_steps)
        r64 = s64.residual(args.ref_fp64_steps)
        eta64, _ = s64.overpotential()
        torch.cuda.synchronize()
        secs64 = time.perf_counter() - t
        s64.close()
        ref = {"fp32_leg": r32, "fp64_leg": {"steps": args.ref_fp64_steps, "residual": r64,
                                               "eta_V": eta64, "seconds": round(secs64, 2)},
               "eta_V": eta64,
               "what": "the chosen form's end state run on in FP32 with extrapolation to residual "
                       f"{args.ref_tol:g}, then {args.ref_fp64_steps} FP64 steps from that field"}
        out["reference"] = ref
        for label in pick:
            e = out[label]["eta_V"]
            rel = abs(e - eta64) / abs(eta64)
            out[label]["eta_rel_err_vs_reference"] = rel
            out[label]["eta_within_1e-4"] = bool(rel <= 1e-4)
    return out


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
    if args.workload == "unet":
        return main_unet(args, ws, rank, local)

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
    s.close()
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

    # the same throughput with 16-bit population storage (the chosen form's
    # storage), one more handle and the same timing
    fp16 = None
    if args.precision == "fp32" and not args.no_fp16_line:
        fp16 = time_steps(L, case, "fp16", args, dist)

    # time to residual 1e-8 (the second half of the metric): plain FP32
    # against the chosen form, each with its clock record, and their
    # overpotentials against a reference steady state
    ttr = None
    if args.time_to_residual > 0 and not args.no_ttr:
        ttr = time_to_residual(L, case, args)

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
        csteps = 10
        cells, wall, procs, planes = oracle_all_cores(args.workload, csteps, 1, args.oracle_procs)
        cpu = {"value": round(cells * 3 * csteps / wall / 1e6, 4), "unit": METRIC,
               "cores": procs * cores_used(), "kind": "oracle",
               "sample": f"{csteps} timed FP64 oracle steps (after 1 untimed) on all {planes} z-planes of "
                         f"the same {case.name} mask, split into {procs} z-slabs (each periodic in z) run "
                         f"concurrently by {procs} single-threaded processes ({cells} fluid cells)"}

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
                                   f"{tinfo.tile_min_blocks} blocks/SM, " + (
                                       "neighbours decoded from per-row fluid bitmasks" if tinfo.neighbour_bits == 1
                                       else f"{tinfo.neighbour_bits}-bit neighbour table") + " (autotuned)",
                           "l2": "state larger than L2 (no flush needed)" if nf * bpc > 129e6 * 2
                           else "state fits in L2"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": args.steps, "fp16_storage": fp16, "time_to_residual": ttr}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def sweep_cases(args, scale=None):
    """The uneven-size sweep: each microstructure at each operating point."""
    from workloads import cases as W
    structs = W.sweep_structures(args.sweep_2d, args.sweep_3d,
                                 scale=args.sweep_scale if scale is None else scale)
    pts = W.sweep_operating_points(args.sweep_points)
    groups = {2: [], 3: []}
    for st in structs:
        for I, x in pts:
            groups[st.dim].append(st.with_(current_A_cm2=I, x_in=x))
    return groups


def extrapolate_every_for(nx):
    """W of the single-mode extrapolation for an anode nx cells long: the
    slowest mode decays as 1/nx^2, so W scales with nx^2 (20,000 steps at
    nx = 256), rounded to 500 steps, at least 1000."""
    return max(1000, int(round(20000 * (nx / 256.0) ** 2 / 500.0)) * 500)


def rre_every(nx):
    """Snapshot spacing W of the reduced-rank extrapolation for an anode nx
    cells long: the slowest mode decays as 1/nx^2, so W scales with nx^2
    (10,000 steps at nx = 256), rounded to 500 steps, at least 1000."""
    return max(1000, int(round(10000 * (nx / 256.0) ** 2 / 500.0)) * 500)


def train_warmstart_net(L, train, tol, args, keep=None, unet=None):
    """Steady states of the training anodes (one batch, FP32 + slowest-mode
    extrapolation) and a warm-start network trained on them; returns the net
    and timings.  With a list `keep`, each training case's dense input volume
    and target (for the PyTorch comparison) are appended to it; with a UNet
    `unet`, each steady state is added to it as a training volume."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nx_max = max(c.solid.shape[2] for c in train)
    b = L.Batch.from_cases(train, precision="fp32", extrapolate_every=extrapolate_every_for(nx_max))
    for k, c in enumerate(train):
        b.set_bc(c.x_in, c.current_A_cm2, case=k)
    n, _, _, st = b.run_to_residual(tol, args.max_steps, raise_on_fail=False)
    net = L.Net(width=704, depth=3, seed=1)
    for k in range(len(train)):
        net.add_sample(b, k)
        if unet is not None:
            unet.add_sample(b, k)
        if keep is not None:
            V = _dense_inputs(net, b, train[k], k)
            X = b.fields(k).astype(np.float32)
            keep.append((V, 100.0 * (X - V[0:3]) * V[16:17]))
    b.close()
    t1 = time.perf_counter()
    loss = net.train(args.ws_iters, batch=8192, lr=args.ws_lr)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, {"data": {"cases": len(train), "rows": net.info()[1], "steps": int(n),
                          "seconds": round(t1 - t0, 2)},
                 "training": {"params": net.info()[0], "iters": args.ws_iters, "batch": 8192, "lr": args.ws_lr,
                              "final_loss": loss, "seconds": round(t2 - t1, 2)}}


# ------------------------------------------------- warm-start comparison
def _dense_inputs(net, handle, case, k):
    """Dense input volume [C, nz, ny, nx] of one case for the convolutional
    comparison: the 16 used feature columns of lbms_net_features scattered
    to the fluid voxels, plus the fluid mask."""
    F = net.features(handle, case.n_fluid, case=k)[:, :16]
    nz, ny, nx = case.solid.shape
    fl = np.flatnonzero(~case.solid.reshape(-1))
    V = np.zeros((17, nz * ny * nx), dtype=np.float32)
    V[:16, fl] = F.T
    V[16, fl] = 1.0
    return V.reshape(17, nz, ny, nx)


def _unet(torch, width=28):
    """A three-level 3-D U-Net (two 3x3x3 convolutions per level, ReLU,
    max-pool down, transposed convolution up, skip concatenation), about
    1M parameters at width 28."""
    nn = torch.nn

    def block(ci, co):
        return nn.Sequential(nn.Conv3d(ci, co, 3, padding=1), nn.ReLU(), nn.Conv3d(co, co, 3, padding=1), nn.ReLU())

    class UNet(nn.Module):
        def __init__(self):
            super().__init__()
            w = width
            self.e1, self.e2, self.e3 = block(17, w), block(w, 2 * w), block(2 * w, 4 * w)
            self.u2 = nn.ConvTranspose3d(4 * w, 2 * w, 2, stride=2)
            self.d2 = block(4 * w, 2 * w)
            self.u1 = nn.ConvTranspose3d(2 * w, w, 2, stride=2)
            self.d1 = block(2 * w, w)
            self.out = nn.Conv3d(w, 3, 1)

        def forward(self, x):
            a = self.e1(x)
            b = self.e2(nn.functional.max_pool3d(a, 2))
            c = self.e3(nn.functional.max_pool3d(b, 2))
            d = self.d2(torch.cat([self.u2(c), b], 1))
            e = self.d1(torch.cat([self.u1(d), a], 1))
            return self.out(e)

    return UNet()


def compare_unet(L, net, kept, test, tol, prec, Wx, modes, args):
    """The convolutional alternative to the pointwise network: a 3-D U-Net
    trained with PyTorch on the same steady states (`kept`: input volumes
    and targets 100 (X - X_profile) on fluid voxels; mean-square error,
    Adam), then used as the start of the same held-out runs.  Returns its
    mean steps and timings."""
    import torch
    dev = torch.device("cuda")
    data = {}
    for V, T in kept:
        data.setdefault(V.shape, []).append((V, T))
    model = _unet(torch).to(dev)
    nparams = sum(p.numel() for p in model.parameters())
    opt = torch.optim.Adam(model.parameters(), lr=1e-3)
    iters = args.ws_iters
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, iters, eta_min=5e-5)
    groups = {sh: (torch.tensor(np.stack([v for v, _ in d]), device=dev),
                   torch.tensor(np.stack([t for _, t in d]), device=dev)) for sh, d in data.items()}
    keys = list(groups)
    gen = torch.Generator(device="cpu").manual_seed(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(iters):
        Vg, Tg = groups[keys[it % len(keys)]]
        idx = torch.randint(0, Vg.shape[0], (min(8, Vg.shape[0]),), generator=gen).to(dev)
        pred = model(Vg[idx])
        m = Vg[idx, 16:17]
        loss = (((pred - Tg[idx]) * m) ** 2).sum() / (3.0 * m.sum())
        opt.zero_grad()
        loss.backward()
        opt.step()
        sched.step()
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    bt = L.Batch.from_cases(test, precision=prec, extrapolate_every=Wx, extrapolate_modes=modes)
    for k, c in enumerate(test):
        bt.set_bc(c.x_in, c.current_A_cm2, case=k)
    torch.cuda.synchronize()
    ta = time.perf_counter()
    with torch.no_grad():
        for k, c in enumerate(test):
            V = _dense_inputs(net, bt, c, k)
            P = model(torch.tensor(V[None], device=dev))[0].cpu().numpy()
            X = np.maximum(V[0:3] + P / 100.0, 1e-6)
            X = X / X.sum(axis=0, keepdims=True)
            bt.set_fields(k, np.where(c.solid[None], 0.0, X))
    torch.cuda.synchronize()
    tb_ = time.perf_counter()
    n, steps, r, st = bt.run_to_residual(tol, args.max_steps, raise_on_fail=False)
    torch.cuda.synchronize()
    tc = time.perf_counter()
    bt.close()
    return {"params": int(nparams), "iters": iters, "final_loss": float(loss.detach()),
            "train_seconds": round(t_train, 2), "mean_steps": float(np.mean(steps)), "max_steps": int(np.max(steps)),
            "converged": bool(np.all(steps > 0)), "start_seconds": round(tb_ - ta, 3),
            "batch_seconds": round(tc - tb_, 2),
            "model": "3-D U-Net, 3 levels, widths 28/56/112, PyTorch convolutions (comparison only)"}


def main_warmstart(args, ws, rank, local):
    """Learned warm start: steady states of seeded 64x32x32 anodes (and, with
    --ws-train-test-shape, of anodes at the held-out grid) from the batched
    solver train the network; on held-out anodes of --ws-test-shape, the
    steps and time to residual 1e-8 from the uniform start, the 1-D profile
    of Section 4.1 and the network's prediction, for the chosen form (FP16
    storage + slowest-mode extrapolation) and, with --ws-plain, plain FP32."""
    import torch
    torch.cuda.set_device(local)
    from paper_1809_01600_gb300 import lbms as L
    from workloads import cases as W
    L.load()
    tol = args.time_to_residual or 1e-8
    nx, ny, nz = (int(v) for v in args.ws_test_shape.split("x"))
    tshape = (nz, ny, nx)
    train = W.warmstart_cases(args.ws_train, 1000)
    if args.ws_train_test_shape:
        train += W.warmstart_cases(args.ws_train_test_shape, 3000, shape=tshape)
    test = W.warmstart_cases(args.ws_test, 5000, shape=tshape)
    out = {"residual": tol, "test_shape": args.ws_test_shape, "train": {"64x32x32": args.ws_train,
                                                                       args.ws_test_shape: args.ws_train_test_shape}}
    kept = [] if args.ws_compare_unet else None
    unet = None
    if args.ws_unet_iters > 0:
        # one batch holds up to 8 volumes of one training grid; one test volume for the start
        def vol(sh):
            return int(np.prod([(d + 3) // 4 * 4 for d in sh]))
        groups = {}
        for c in train:
            groups[c.solid.shape] = groups.get(c.solid.shape, 0) + 1
        vmax = max([min(8, n) * vol(sh) for sh, n in groups.items()] + [vol(tshape)])
        unet = L.UNet(width=args.ws_unet_width, max_voxels=vmax, seed=1)
    net, info = train_warmstart_net(L, train, tol, args, keep=kept, unet=unet)
    out.update(info)
    if unet is not None:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        uloss = unet.train(args.ws_unet_iters, max_batch=8, lr=args.ws_lr)
        torch.cuda.synchronize()
        out["unet_training"] = {"params": unet.info()[0], "iters": args.ws_unet_iters, "max_batch": 8,
                                "lr": args.ws_lr, "final_loss": uloss,
                                "seconds": round(time.perf_counter() - t0, 2),
                                "max_voxels": unet.max_voxels,
                                "model": "3-D U-Net, 3 levels, widths %d/%d/%d, implicit-GEMM tcgen05 convolutions of this "
                                         "project" % (args.ws_unet_width, 2 * args.ws_unet_width,
                                                      4 * args.ws_unet_width)}
    Wx = extrapolate_every_for(nx)
    forms = [("fp16_extrapolated", "fp16", Wx, 1)]
    if args.ws_plain:
        forms.insert(0, ("plain_fp32", "fp32", 0, 1))
    for label, prec, Wx, modes in forms:
        res = {"extrapolate_every": Wx, "extrapolate_modes": modes}
        starts = [st for st in args.ws_starts.split(",") if st and (st != "unet" or unet is not None)]
        for start in starts:
            bt = L.Batch.from_cases(test, precision=prec, extrapolate_every=Wx, extrapolate_modes=modes,
                                    init_mode="profile1d" if start == "profile1d" else "uniform")
            for k, c in enumerate(test):
                bt.set_bc(c.x_in, c.current_A_cm2, case=k)
            torch.cuda.synchronize()
            clocks = ClockSampler(torch.cuda.current_device())
            clocks.start()
            ta = time.perf_counter()
            if start == "network":
                for k in range(len(test)):
                    net.warm_start(bt, k)
            elif start == "unet":
                for k in range(len(test)):
                    unet.warm_start(bt, k)
            torch.cuda.synchronize()
            tb = time.perf_counter()
            n, steps, r, st = bt.run_to_residual(tol, args.max_steps, raise_on_fail=False)
            torch.cuda.synchronize()
            tc = time.perf_counter()
            res[start] = {"mean_steps": float(np.mean(steps)), "max_steps": int(np.max(steps)),
                          "converged": bool(np.all(steps > 0)), "start_seconds": round(tb - ta, 3),
                          "batch_seconds": round(tc - tb, 2), "clocks": clocks.stop()}
            bt.close()
        if args.ws_compare_unet and label == "fp16_extrapolated":
            res["unet_pytorch"] = compare_unet(L, net, kept, test, tol, prec, Wx, modes, args)
        for start in ("profile1d", "network", "unet", "unet_pytorch"):
            if start in res and "uniform" in res:
                res[start]["steps_vs_uniform"] = round(res[start]["mean_steps"] / res["uniform"]["mean_steps"], 3)
        out[label] = res
    tc, ms = net.gemm_calls()
    out["gemm_calls"] = {"tcgen05": tc, "mma_sync": ms}
    net.close()
    if unet is not None:
        out["unet_gemm_calls"] = {"tcgen05": unet.gemm_calls()}
        unet.close()
    if rank == 0:
        res0 = out["fp16_extrapolated"]
        chosen = next(c for c in ("unet", "network", "profile1d", "uniform") if c in res0)
        v = res0[chosen]["mean_steps"]
        line = {"metric": "steps to residual (held-out anodes, %s start, FP16 + extrapolation)"
                          % {"unet": "U-Net", "network": "network"}.get(chosen, chosen), "value": v,
                "unit": "steps", "n_gpus": 1, "higher_is_better": False, "vs_baseline": None,
                "dtype": "bf16 network, f32 LBM", "data": "synthetic",
                "config": {"workload": f"learned warm start, {len(train)} training anodes "
                                       f"({args.ws_train} 64x32x32 + {args.ws_train_test_shape} "
                                       f"{args.ws_test_shape}) and {len(test)} held-out {args.ws_test_shape} "
                                       f"D3Q19 anodes"},
                "warm_start": out}
        print(json.dumps(line))
    return 0


def _unet_volumes(n, shape, seed=7):
    """n synthetic training volumes like the warm-start inputs: 16 feature
    channels in [0, 1] on fluid voxels (porosity 0.45), the fluid mask, and
    targets that are a smooth function of them (zero on solid voxels)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        m = (rng.random((1, nz, ny, nx)) < 0.45).astype(np.float32)
        x = np.concatenate([rng.random((16, nz, ny, nx)).astype(np.float32) * m, m], axis=0)
        t = ((3.0 * x[0:3] - 1.0) * x[3:4] + x[4:7]) * m
        out.append((x, t.astype(np.float32)))
    return out


def main_unet(args, ws, rank, local):
    """Training-step time of the 3-D U-Net on this project's kernels
    (implicit-GEMM tcgen05 convolutions) over --unet-batch synthetic volumes
    of --unet-shape already on the device; with --unet-torch, the same
    network and volumes with PyTorch convolutions (TF32, and BF16 autocast)."""
    import torch
    torch.cuda.set_device(local)
    from paper_1809_01600_gb300 import lbms as L
    L.load()
    nx, ny, nz = (int(v) for v in args.unet_shape.split("x"))
    B, K, W = args.unet_batch, args.unet_steps, max(args.warmup, 3)
    vols = _unet_volumes(B, (nz, ny, nx))
    u = L.UNet(width=args.ws_unet_width, max_voxels=B * nx * ny * nz, seed=1)
    for x, t in vols:
        u.add_volume(x, t)
    u.train(W, max_batch=B, lr=args.ws_lr)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0 = u.gemm_calls()
    e0.record()
    loss = u.train(K, max_batch=B, lr=args.ws_lr)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    clk = clocks.stop()
    gemms = (u.gemm_calls() - c0) // K
    u.close()
    out = {"metric": "3-D U-Net training step (this project's kernels)", "value": round(ms, 3), "unit": "ms/step",
           "n_gpus": 1, "steps": K, "warmup": W, "higher_is_better": False, "vs_baseline": None,
           "dtype": "bf16 (fp32 accumulation, fp32 master weights)", "data": "synthetic",
           "config": {"workload": f"U-Net width {args.ws_unet_width}, {B} volumes of {args.unet_shape} per step",
                      "tcgen05_products_per_step": int(gemms), "final_loss": loss},
           "clocks": clk}
    if args.unet_torch:
        dev = torch.device("cuda")
        xs = torch.tensor(np.stack([x for x, _ in vols]), device=dev)
        ts = torch.tensor(np.stack([t for _, t in vols]), device=dev)
        m = xs[:, 16:17]
        for amp in (False, True):
            torch.manual_seed(0)
            model = _unet(torch, args.ws_unet_width).to(dev)
            opt = torch.optim.Adam(model.parameters(), lr=args.ws_lr)

            def step():
                with torch.autocast("cuda", dtype=torch.bfloat16, enabled=amp):
                    pred = model(xs)
                lo = (((pred.float() - ts) * m) ** 2).sum() / (3.0 * m.sum())
                opt.zero_grad()
                lo.backward()
                opt.step()
            for _ in range(W):
                step()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(K):
                step()
            e1.record()
            torch.cuda.synchronize()
            out["pytorch_bf16_autocast_ms" if amp else "pytorch_tf32_ms"] = round(e0.elapsed_time(e1) / K, 3)
            del model, opt
    if rank == 0:
        print(json.dumps(out))
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


BATCH_MAX_CELLS = 100_000_000   # a batch's link offsets (link x row stride) stay 32-bit for D3Q19


def _batched_steps(L, groups, precision, steps, warmup, stream, dist):
    """The cases of each lattice group in as few batches as the step
    kernel's 32-bit in-species offsets allow (at most BATCH_MAX_CELLS fluid
    cells each; one launch per batch and step); CUDA-event time of `steps`
    steps over all batches."""
    import torch
    batches = []
    for dim in (2, 3):
        chunk, cells = [], 0
        for c in groups[dim] + [None]:
            if c is not None and (not chunk or cells + c.n_fluid <= BATCH_MAX_CELLS):
                chunk.append(c)
                cells += c.n_fluid
                continue
            if chunk:
                b = L.Batch.from_cases(chunk, precision=precision)
                for k, cc in enumerate(chunk):
                    b.set_bc(cc.x_in, cc.current_A_cm2, case=k)
                batches.append((dim, chunk, b))
            chunk, cells = ([c], c.n_fluid) if c is not None else ([], 0)
    for _, _, b in batches:
        b.step(warmup)
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
        b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    tiles = ["%dD x%d: %d cells, %d blocks/SM, nb%d" % (dim, len(cs), b.info().tile_cells, b.info().tile_min_blocks,
                                                         b.info().neighbour_bits) for dim, cs, b in batches]
    etas = [b.overpotentials(raise_on_fail=False)[0] for _, _, b in batches]
    for _, _, b in batches:
        b.close()
    return ms, clk, tiles, etas, len(batches)


def _sequential_steps(L, groups, precision, steps, stream):
    """The same cases, one handle each, stepped one after another: summed
    CUDA-event time of `steps` steps per handle."""
    import torch
    t = 0.0
    for dim in (2, 3):
        for c in groups[dim]:
            s = L.Solver.from_case(c, precision=precision)
            s.set_bc(c.x_in, c.current_A_cm2)
            s.step(32)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            s.step(steps)
            a1.record(stream)
            torch.cuda.synchronize()
            t += a0.elapsed_time(a1) / 1e3
            s.close()
    return t


def main_sweep(args, ws, rank, local):
    """The batched sweep: --sweep-2d 2-D and --sweep-3d 3-D seeded
    microstructures of uneven size, each at --sweep-points operating points,
    one launch per lattice and step (batched, autotuned tile).  Then the
    same recipe with grids scaled by --sweep-small-scale, where the cases are
    small enough that one launch per case leaves the GPU idle: batched
    against one handle per case."""
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1809_01600_gb300 import lbms as L
    L.load()
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    groups = sweep_cases(args)
    t_gen = time.perf_counter() - t_gen
    nf = sum(c.n_fluid for d in (2, 3) for c in groups[d])
    ms, clk, tiles, etas, nlaunch = _batched_steps(L, groups, args.precision, args.steps, args.warmup, stream, dist)
    t_dev = max_over_ranks(dist, ms / 1e3, "cuda")
    units = nf * 3 * args.steps * ws
    value = units / t_dev / 1e6
    bpc = {d: bytes_per_cell(d, args.precision) for d in (2, 3)}
    alg = sum(c.n_fluid * bpc[c.dim] for d in (2, 3) for c in groups[d])
    achieved = alg / (t_dev / args.steps) / 1e9
    peak, peak_kind = measured_peak_hbm()
    eta_all = np.concatenate([np.asarray(e) for e in etas])

    small = None
    if args.sweep_small_scale > 0:
        sg = sweep_cases(args, scale=args.sweep_small_scale)
        snf = sum(c.n_fluid for d in (2, 3) for c in sg[d])
        sms, sclk, stiles, _, _ = _batched_steps(L, sg, args.precision, args.steps, args.warmup, stream, None)
        seq_steps = max(1, min(args.steps, 200))
        t_seq = _sequential_steps(L, sg, args.precision, seq_steps, stream)
        bval = snf * 3 * args.steps / (sms / 1e3) / 1e6
        sval = snf * 3 * seq_steps / t_seq / 1e6
        small = {"cases": {"2d": len(sg[2]), "3d": len(sg[3])}, "fluid_cells": snf,
                 "scale": args.sweep_small_scale, "batched": {"value": round(bval, 2), "unit": METRIC,
                                                              "ms_per_step": round(sms / args.steps, 5),
                                                              "tiles": stiles, "clocks": sclk},
                 "sequential": {"value": round(sval, 2), "unit": METRIC, "steps": seq_steps,
                                "what": "the same cases, one handle each, stepped one after another"},
                 "speedup_vs_sequential": round(bval / sval, 2)}
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
                           "launches_per_step": nlaunch, "host_generation_seconds": round(t_gen, 1)},
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_kind},
                "small_cases": small,
                "eta_V_range": [float(np.nanmin(eta_all)), float(np.nanmax(eta_all))],
                "clocks": clk, "gpu_launches": args.steps * nlaunch}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main_reference(args, ws, rank):
    """The oracle arm: the FP64 CPU oracle timed on every host core, one
    process per z-slab of the same workload, bounded to about 150 s; with
    --oracle-ttr, the oracle's own time to residual on the workload (one
    process: a single small case)."""
    if rank != 0:
        return 0
    case = make_case(args.workload)
    nz = case.solid.shape[0]
    procs = max(1, min(args.oracle_procs or os.cpu_count() or 1, nz))
    probe = case.with_(solid=np.ascontiguousarray(case.solid[:1]))
    t_plane = run_oracle(probe, 1, 1)                  # seconds per z-plane and step
    per_proc = max(1, int(150.0 / max(t_plane * (args.steps + args.warmup), 1e-9)))
    planes = min(nz, procs * per_proc)
    cells, wall, procs, planes = oracle_all_cores(args.workload, args.steps, args.warmup, procs, planes)
    value = cells * 3 * args.steps / wall / 1e6
    desc = (f"FP64 CPU oracle, {args.steps} timed steps (after {args.warmup}) on the first {planes} of "
            f"{nz} z-planes of the {case.name} mask ({cells} fluid cells), split into {procs} z-slabs "
            f"(each periodic in z) run concurrently by {procs} single-threaded processes")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": METRIC,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(wall / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case.name, "precision": args.precision,
                       "parallelism": f"{procs} host cores"},
            "cpu_baseline": {"value": round(value, 4), "unit": METRIC, "cores": procs * cores_used(),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 4), "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    if args.oracle_ttr:
        from oracle import Oracle
        o = Oracle(case)
        t = time.perf_counter()
        n, r = o.run_to_residual(args.time_to_residual or 1e-8, args.max_steps, 100)
        secs = time.perf_counter() - t
        line["time_to_residual"] = {"tol": args.time_to_residual or 1e-8, "steps": int(n), "residual": r,
                                    "seconds": round(secs, 2), "eta_V": o.overpotential(), "cores": 1,
                                    "what": "the FP64 oracle run to the residual on the whole workload "
                                            "from the uniform inlet start (one process)"}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
