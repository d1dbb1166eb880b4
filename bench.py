"""Benchmark: sink-site contractions per second of the 3He correlator at 24^3 x 48.

One step = one evaluation of the correlator C(t) of the 3He_II-s operator (the stand-in
for the printed 3He_II, which vanishes identically) over every sink site of a 24^3 x 48
lattice (663552 sink-site contractions), with the e-graph plan in the FP32 arithmetic with
its error guards (MBC_PREC_FP32: complex FP32 minors and contraction, compensated sums,
the time slices whose estimated C(t) error exceeds 1e-6 recomputed in double-float):
staging, minors, contraction, guard, recompute and the site sum, all in the library's
kernels.  Inputs (2 x 1.5 GB of complex double propagators, generated on the GPU by the
seeded recipe of mbc_inputs) are resident in HBM and larger than L2.

Prints one JSON line (rank 0).  Extra keys: the roofline of the dominant kernel (timed
alone, guards off), the FP64 and double-float plans on a subset of time slices (same
metric, timed over repeats) with the FP32 C(t) error against the FP64 C(t), per-site
errors against the oracle on the sampled sites of the CPU baseline, the oracle timed on
the host cores (cpu_baseline), an end-to-end figure through the host-buffer entry point,
SM clocks sampled during the timed region and the number of kernel launches.
``--impl reference`` times the oracle instead (on a bounded sample).
"""
from __future__ import annotations

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

METRIC = "sink-site contractions/sec (He-3 II, 24^3x48), FP64 vs mixed, % FLOP peak"
UNIT = "contractions/s"
OPERATOR = "he3_II_s"
L, T = 24, 48
SEED, KAPPA = 3, 0.5
SM_COUNT = 152
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (4 sub-partitions x 32)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


FP64_FMA_PER_SM = 2              # DFMA per cycle per SM (ncu: sm__sass_thread_inst_executed_op_dfma peak)


def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak from unit counts and clock: SMs x lanes x 2 flop x clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def fp64_peak_tflops(sm_mhz):
    """FP64 FMA peak from unit counts and clock: SMs x DFMA/cycle x 2 flop x clock."""
    return SM_COUNT * FP64_FMA_PER_SM * 2 * sm_mhz * 1e6 / 1e12


KERNEL_SOURCES = ("egraph32.cu", "numeric.cuh", "common.cuh", "device.cuh", "walk.hpp")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "egraph32_kernel_he3_II_s_24x48.md")
BLOCK_SOURCES = ("blocks.cu", "blocks.cuh", "numeric.cuh", "common.cuh", "device.cuh")
BLOCK_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "block_kernels_he3_II_s_24x48.md")


def kernel_hash(sources=KERNEL_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2201_04269_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic_per_site(path=TRAFFIC_FILE, sources=KERNEL_SOURCES):
    """DRAM bytes per site from the committed ncu summary, if the kernel sources are
    unchanged since it was taken (else None)."""
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if line.startswith("kernel_source_hash:"):
            vals["hash"] = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_site:"):
            vals["bytes"] = float(line.split(":", 1)[1].strip())
    if vals.get("hash") != kernel_hash(sources) or "bytes" not in vals:
        return None
    return vals["bytes"]


def fields(set_index, t_list=None, seed=SEED, kappa=KAPPA, noise=None, lat=None):
    import mbc_inputs as mi
    Ls, Ts = lat or (L, T)
    U = mi.propagator_field(seed, set_index, 0, Ts, Ls ** 3, kappa, noise, t_list)
    D = mi.propagator_field(seed, set_index, 1, Ts, Ls ** 3, kappa, noise, t_list)
    return U, D


def device_fields(set_indices, t_list, seed, kappa, noise, Ls):
    """U, D cuda complex128 [n_sets, n_t, L^3, 12, 12] generated on the GPU by the seeded
    recipe of mbc_inputs (the same entries as fields(), up to the last bits of the GPU's
    transcendental functions)."""
    import torch
    import mbc_inputs as mi
    V3 = Ls ** 3
    U = torch.empty(len(set_indices), len(t_list), V3, 12, 12, dtype=torch.complex128, device="cuda")
    D = torch.empty_like(U)
    st = torch.cuda.current_stream().cuda_stream
    for k, si in enumerate(set_indices):
        mi.fill_device(U[k].data_ptr(), seed, si, 0, V3, t_list, kappa, noise, st)
        mi.fill_device(D[k].data_ptr(), seed, si, 1, V3, t_list, kappa, noise, st)
    torch.cuda.synchronize()
    return U, D


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(n_sites_target=None, seconds=20.0):
    """The oracle (canonical form, plain C, OpenMP over sites) on a bounded sample of
    the same workload: sites spread over the time slices."""
    from oracle import correlator as ocor
    from oracle import native
    from oracle import operators as oops
    import mbc_inputs as mi
    native.build()
    plan = ocor.CanonicalPlan(oops.build(OPERATOR))
    threads = native.max_threads()
    rng = np.random.default_rng(0)
    # calibrate on a few sites, then size the sample to ~`seconds` of wall time
    probe = [(t, int(rng.integers(L ** 3))) for t in rng.choice(T, size=max(8 * threads, 16))]

    def regen(pts):
        U = np.concatenate([mi.site_matrices(SEED, 0, 0, t, [x], KAPPA) for t, x in pts])
        D = np.concatenate([mi.site_matrices(SEED, 0, 1, t, [x], KAPPA) for t, x in pts])
        return U, D

    U, D = regen(probe)
    plan.site_values(U[:threads], D[:threads], n_threads=threads)      # warm-up (threads, first-call costs)
    t0 = time.perf_counter()
    plan.site_values(U, D, n_threads=threads)
    dt = time.perf_counter() - t0
    n = n_sites_target or max(threads, int(seconds / max(dt / len(probe), 1e-9)))
    pts = [(int(t), int(rng.integers(L ** 3))) for t in rng.integers(0, T, size=n)]
    U, D = regen(pts)
    t0 = time.perf_counter()
    vals = plan.site_values(U, D, n_threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} random sink sites of {OPERATOR} {L}^3x{T} (canonical merged form, plain C, "
                      f"OpenMP over sites), {dt:.1f} s"}, dt, (pts, vals)


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = []
    meta = None
    for i in range(args.warmup + args.steps):
        meta, dt, _ = cpu_baseline(seconds=min(20.0, 100.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            steps.append(dt)
    value = meta["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{OPERATOR} (stand-in for He-3 II) {L}^3x{T}, 1 source(s) per GPU",
                       "algorithm": "oracle (canonical merged form, plain C, OpenMP over sites) on a bounded sample "
                                    "of the workload's sites", "arithmetic": "fp64"},
            "cpu_baseline": meta, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_blocks(args, rank, world, local):
    """The block form (Secs. 2-4): every sink baryon projected to zero momentum, blocks of
    every sink site, then the block factor tree per time slice; FP64.  Same workload
    shape as the headline; a step covers every sink site of every slice."""
    import torch
    import torch.distributed as dist
    from paper_2201_04269_gb300 import Context, shard

    Lb, Tb = (int(v) for v in args.lattice.split("x"))
    t_list = list(range(Tb)) if args.slices <= 0 else [int(t) for t in np.linspace(0, Tb - 1, args.slices).round()]
    sets = list(shard.local_sets(args.sets * world, rank, world))
    hs = [fields(si, t_list, args.seed, args.kappa, args.noise, (Lb, Tb)) for si in sets]
    U_h = np.stack([h[0] for h in hs])
    D_h = np.stack([h[1] for h in hs])
    del hs
    n_sets, n_t, n_v = U_h.shape[:3]
    n_sites = n_sets * n_t * n_v
    stream = torch.cuda.current_stream()
    U = torch.from_numpy(U_h).cuda()
    D = torch.from_numpy(D_h).cuda()
    C = torch.zeros(n_sets, n_t, dtype=torch.complex128, device="cuda")
    ctx = Context(local)
    local_form = args.algo == "blocks_local"
    plan = ctx.block_plan(args.op, "fp64" if local_form else args.prec)
    info = plan.info

    def step():
        if local_form:
            plan.correlator_local(U, D, C, stream=stream)
        else:
            plan.correlator(U, D, C, Lb, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = ctx.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = ctx.launches - launches0
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    clocks = clk.summary()
    sm_max = measured_peaks().get("sm_max_mhz", 2070.0)
    prec = "fp64" if local_form else args.prec
    # the local form walks the whole block tree at every site
    flops = (info["block_flops_per_site"] * n_sites +
             info["tree_flops_per_slice"] * (n_sites if local_form else n_sets * n_t))
    achieved = flops / (ms * 1e-3) / 1e12
    peak = fp64_peak_tflops(sm_max) if prec == "fp64" else fp32_peak_tflops(sm_max)
    headline_shape = (args.op == OPERATOR and (Lb, Tb) == (L, T) and args.slices <= 0 and args.sets == 1)
    tps = recorded_traffic_per_site(BLOCK_TRAFFIC_FILE, BLOCK_SOURCES) if headline_shape and not local_form else None
    # end to end: pinned host fields copied in, C copied out, inside the timed region
    U_pin = torch.from_numpy(U_h).pin_memory()
    D_pin = torch.from_numpy(D_h).pin_memory()
    C_pin = torch.zeros(n_sets, n_t, dtype=torch.complex128).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U.copy_(U_pin, non_blocking=True)
    D.copy_(D_pin, non_blocking=True)
    step()
    C_pin.copy_(C, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if rank == 0:
        form = "local sink" if local_form else "zero-momentum projected blocks"
        line = {"metric": f"sink-site contractions/sec ({args.op} block form, {form}, {Lb}^3x{Tb}, {prec})",
                "value": world * n_sites / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32x2" if prec == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": f"{args.op} {Lb}^3x{Tb}" + (f" ({n_t} slices)" if n_t != Tb else "") +
                                       f", {n_sets} source(s) per GPU, block form ({form}), {prec}",
                           "sites_per_gpu": n_sites,
                           "l2": f"inputs {2 * U_h.nbytes / 1e9:.2f} GB per GPU" +
                                 (", larger than L2" if 2 * U_h.nbytes > 129e6 else ", smaller than L2"),
                           "block_plan": {k: info[k] for k in ("n_w", "expanded_terms", "merged_terms", "factors",
                                                               "level_nodes")}},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None if tps is None else tps * n_sites,
                             "kernel": ("block_local_kernel" if local_form else
                                        "block_project_kernel + block_tree_kernel"),
                             "kernel_source_hash": kernel_hash(BLOCK_SOURCES),
                             "flops_per_site": info["block_flops_per_site"],
                             "tree_flops_per_slice": info["tree_flops_per_slice"],
                             "peak_basis": (f"FP64: {SM_COUNT} SMs x {FP64_FMA_PER_SM} DFMA/cycle x 2 x {sm_max:.0f} MHz "
                                            "(derived)" if prec == "fp64" else
                                            f"FP32: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz "
                                            "(derived)")},
                "cpu_baseline": None,
                "e2e": {"value": world * n_sites / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(2 * U_h.nbytes),
                        "d2h_bytes_per_step": int(C_pin.numel() * 16)},
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.destroy()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mbc", choices=["mbc", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--no-kernel", action="store_true",
                    help="skip timing the FP32 kernel alone (the roofline then uses the whole step)")
    ap.add_argument("--fp64-slices", type=int, default=6)
    # other workloads and algorithms (the default is the benchmark's headline configuration)
    ap.add_argument("--op", default=OPERATOR)
    ap.add_argument("--algo", default="egraph", choices=["egraph", "tree", "direct", "blocks", "blocks_local"],
                    help="blocks = hadron blocks projected to zero momentum and the block factor tree; "
                         "blocks_local = the block form of the local-sink correlator (FP64)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "mixed", "fp64"],
                    help="fp32 = FP32 with error guards (default), mixed = double-float, fp64")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the plan's default schedule (default: mbc_autotune on two slices first)")
    ap.add_argument("--guard", type=float, default=None, help="FP32 error-estimate threshold (default: the plan's)")
    ap.add_argument("--lattice", default=f"{L}x{T}", help="L x T, e.g. 16x32")
    ap.add_argument("--slices", type=int, default=0, help="time slices evaluated (0 = all)")
    ap.add_argument("--sites", type=int, default=0, help="sink sites per slice (0 = all)")
    ap.add_argument("--sets", type=int, default=1, help="propagator sets (source times) per GPU")
    ap.add_argument("--seed", type=int, default=SEED)
    ap.add_argument("--kappa", type=float, default=KAPPA)
    ap.add_argument("--noise", type=float, default=None)
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched 64-set workload (timed with the headline on one GPU)")
    ap.add_argument("--batched-sets", type=int, default=64, help="propagator sets of the batched workload")
    ap.add_argument("--save-c", default=None, help="write the timed run's C(t) [sets, T] to this .npy file")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2201_04269_gb300 import Context, build

    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()

    if args.algo in ("blocks", "blocks_local"):
        run_blocks(args, rank, world, local)
        if world > 1:
            dist.destroy_process_group()
        return

    run_local(args, rank, world, local)
    if world > 1:
        dist.destroy_process_group()


def timed(fn, reps, stream):
    """Average ms of reps calls of fn, CUDA events on the stream (one warm-up call first)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


BATCHED_OPS = ("proton", "dinucleon_I", "dinucleon_II", "he3_I", "he3_II")


def run_batched(local, stream, n_sets=64):
    """The batched workload: 64 propagator sets (16 configurations x 4 source times; sets
    0-31 on 16^3 x 32, 32-63 on 24^3 x 48, about 117 GB generated on the GPU) x the five
    operators of Eq. 2 and the proton, FP32 e-graph plans with their guards, all 320 items
    in one mbc_batch (one persistent FP32 launch over every (item, site) unit, the slice
    guard, the double-float recompute, the site sums) captured in a CUDA graph and timed
    over one replay (a step takes minutes; the capture itself loads the kernels and the
    reservation sizes every buffer, so there is no untimed warm-up).  The vanishing D_II
    and He-3 II items cost nothing; their sites are reported apart.  n_sets < 64 takes the
    first n_sets / 2 sets of each lattice."""
    import torch
    import mbc_inputs as mi
    from paper_2201_04269_gb300 import Context, abi
    w = mi.WORKLOADS["batched_64"]
    ctx = Context(local)
    plans = {op: ctx.plan_operator(op, "egraph", "fp32") for op in BATCHED_OPS}
    items, keep = [], []
    st = stream.cuda_stream
    live = dead = 0
    half = w["sets"] // 2
    for s in [k for k in range(w["sets"]) if k % half < n_sets // 2]:
        Lb, Tb = (w["L"][0], w["T"][0]) if s < half else (w["L"][1], w["T"][1])
        V3 = Lb ** 3
        U = torch.empty(1, Tb, V3, 12, 12, dtype=torch.complex128, device="cuda")
        D = torch.empty_like(U)
        mi.fill_device(U.data_ptr(), w["seed"] + s, s, 0, V3, list(range(Tb)), w["kappa"], None, st)
        mi.fill_device(D.data_ptr(), w["seed"] + s, s, 1, V3, list(range(Tb)), w["kappa"], None, st)
        keep += [U, D]
        for op in BATCHED_OPS:
            C = torch.zeros(1, Tb, dtype=torch.complex128, device="cuda")
            keep.append(C)
            items.append(dict(plan=plans[op].handle, U=U, D=D, C=C, site_out=None, n_sets=1, T=Tb, V3=V3))
            if plans[op].info["canonical_terms"]:
                live += Tb * V3
            else:
                dead += Tb * V3
    field_bytes = sum(k.numel() * 16 for k in keep if k.dim() == 5)
    abi.mbc_batch_reserve(ctx.handle, items)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    n0 = ctx.launches
    with torch.cuda.graph(g, stream=cap):
        ctx.batch(items, stream=torch.cuda.current_stream())
    launches = ctx.launches - n0                      # the kernels the graph holds
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    recomputed = ctx.fp32_recomputed
    out = {"workload": f"batched: {n_sets} propagator sets ({n_sets // 2} on 16^3x32, {n_sets // 2} on 24^3x48) x "
                       f"proton, dinucleon I/II, He-3 I/II = {len(items)} items, FP32 e-graph plans with guards, "
                       "one mbc_batch captured in a CUDA graph",
           "value": live / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": 1, "warmup": 0,
           "contractions_per_step": live, "vanishing_sites_per_step": dead,
           "fields_gb": field_bytes / 1e9, "kernel_launches_per_step": launches,
           "recomputed_sites_per_step": recomputed, "recomputed_fraction": recomputed / max(1, live),
           "clocks": clk.summary()}
    del g
    for p in plans.values():
        p.destroy()
    ctx.close()
    del keep
    torch.cuda.empty_cache()
    return out


def run_local(args, rank, world, local):
    """The local-sink correlator (e-graph, tree or direct plan) on the GPU."""
    import torch
    import torch.distributed as dist
    from paper_2201_04269_gb300 import Context, shard

    stream = torch.cuda.current_stream()
    # weak scaling: every rank evaluates its own propagator sets (its own source times)
    Lb, Tb = (int(v) for v in args.lattice.split("x"))
    t_list = list(range(Tb)) if args.slices <= 0 else [int(t) for t in np.linspace(0, Tb - 1, args.slices).round()]
    sets = list(shard.local_sets(args.sets * world, rank, world))
    U, D = device_fields(sets, t_list, args.seed, args.kappa, args.noise, Lb)
    if args.sites > 0:
        U, D = U[:, :, :args.sites].contiguous(), D[:, :, :args.sites].contiguous()
    n_sets, n_t, n_v = U.shape[:3]
    n_sites = n_sets * n_t * n_v
    field_bytes = 2 * U.numel() * 16
    C = torch.zeros(n_sets, n_t, dtype=torch.complex128, device="cuda")
    ctx = Context(local)
    plan = ctx.plan_operator(args.op, args.algo, args.prec)
    if args.guard is not None:
        plan.set_guard(args.guard, float("inf") if args.guard == float("inf") else None)
    info = plan.info
    fp32 = args.prec == "fp32"
    headline = (args.op == OPERATOR and args.algo == "egraph" and args.prec == "fp32" and (Lb, Tb) == (L, T)
                and args.slices <= 0 and args.sites <= 0 and args.sets == 1 and args.noise is None
                and args.guard is None)
    tuned = None
    if not args.no_autotune and args.algo == "egraph":
        from paper_2201_04269_gb300 import abi
        default_schedule = abi.mbc_get_schedule(plan.handle)
        t0 = time.perf_counter()
        tuned = {"default": default_schedule,
                 "tuned": plan.autotune(U, D, min(n_sites, 2 * n_v), stream=stream),
                 "tuning_sites": min(n_sites, 2 * n_v), "tuning_s": round(time.perf_counter() - t0, 2)}

    def step():
        plan.correlator(U, D, C, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = ctx.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = ctx.launches - launches0
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        ms = float(t.item())
    clocks = clk.summary()
    C_main = C.cpu().numpy().copy()
    if args.save_c and rank == 0:
        np.save(args.save_c, C_main)
    recomputed = ctx.fp32_recomputed if fp32 else 0
    guards = plan.guard if fp32 else None

    # the dominant kernel alone: for FP32 plans with both guards off (no recompute, no slice
    # guard), so that the step is the FP32 kernel and the site sum
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    if fp32 and not args.no_kernel:
        plan.set_guard(float("inf"), float("inf"))
        ms_kernel = timed(step, max(1, min(args.steps, 3)), stream)
        plan.set_guard(*guards)
        kname = "egraph32_kernel"
    elif fp32:
        ms_kernel = ms
        kname = "egraph32_kernel (whole step: guard, recompute and site sum included)"
    else:
        ms_kernel = ms
        kname = {"egraph": "egraph_kernel", "tree": "minor_table_kernel + tree_walk_kernel",
                 "direct": "direct_kernel"}[args.algo] + ("<MIXED>" if args.prec == "mixed" else "<FP64>")
    achieved = info["flops_per_site"] * n_sites / (ms_kernel * 1e-3) / 1e12
    peak = fp64_peak_tflops(sm_max) if args.prec == "fp64" else fp32_peak_tflops(sm_max)
    tps = recorded_traffic_per_site() if headline else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None if tps is None else tps * n_sites, "kernel": kname,
                "kernel_ms": ms_kernel, "kernel_source_hash": kernel_hash(),
                "flops_per_site": info["flops_per_site"], "flop_model": "8 flop per complex multiply-add of the plan",
                "peak_basis": (f"FP64: {SM_COUNT} SMs x {FP64_FMA_PER_SM} DFMA/cycle x 2 x {sm_max:.0f} MHz (derived)"
                               if args.prec == "fp64" else
                               f"FP32: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz (derived)")}

    # the FP64 and double-float plans on a subset of time slices (same metric), timed over
    # repeats; the main plan's C(t) against the FP64 C(t) on those slices
    compare = {}
    if args.fp64_slices > 0 and args.algo == "egraph" and args.prec != "fp64":
        ts = sorted(set(np.linspace(0, n_t - 1, min(args.fp64_slices, n_t)).round().astype(int).tolist()))
        Us, Ds = U[:1, ts].contiguous(), D[:1, ts].contiguous()
        n_sub = len(ts) * n_v
        reps = max(1, min(args.steps, 5))
        c64 = None
        for prec in ("fp64", "mixed") if fp32 else ("fp64",):
            p2 = ctx.plan_operator(args.op, "egraph", prec)
            Cs = torch.zeros(1, len(ts), dtype=torch.complex128, device="cuda")
            with Clocks(local) as clk2:
                ms2 = timed(lambda: p2.correlator(Us, Ds, Cs, stream=stream), reps, stream)
            cs = Cs.cpu().numpy()[0]
            tf = p2.info["flops_per_site"] * n_sub / (ms2 * 1e-3) / 1e12
            entry = {"value": n_sub / (ms2 * 1e-3), "unit": UNIT, "time_slices": ts, "repeats": reps,
                     "tflops": tf, "clocks_sm_mhz": clk2.summary()["sm_mhz"],
                     "speedup_of_main": (n_sites / (ms * 1e-3)) / (n_sub / (ms2 * 1e-3))}
            if prec == "fp64":
                entry["frac_fp64_peak"] = tf / fp64_peak_tflops(sm_max)
                c64 = cs
            compare[prec] = entry
            p2.destroy()
        cm = C_main[0][ts]
        compare["rel_err_vs_fp64"] = {
            "max_over_t": float(np.max(np.abs(cm - c64) / np.maximum(np.abs(c64), 1e-300))),
            "normwise": float(np.max(np.abs(cm - c64)) / np.max(np.abs(c64)))}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        U_pin = torch.empty(U.shape, dtype=U.dtype).pin_memory()
        D_pin = torch.empty(D.shape, dtype=D.dtype).pin_memory()
        U_pin.copy_(U)
        D_pin.copy_(D)
        C_pin = torch.zeros(n_sets, n_t, dtype=torch.complex128).pin_memory()
        plan.correlator_host(U_pin, D_pin, C_pin, stream=stream)
        t0 = time.perf_counter()
        plan.correlator_host(U_pin, D_pin, C_pin, stream=stream)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * n_sites / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(U_pin.numel() * 16 * 2),
               "d2h_bytes_per_step": int(C_pin.numel() * 16)}
        del U_pin, D_pin

    cpu, accuracy = None, None
    if rank == 0 and world == 1 and headline and not args.no_cpu:
        cpu, _, (pts, ref) = cpu_baseline()
        # per-site values of the headline plan (per-site guard active) on the sampled sites
        S = torch.zeros(n_sets, n_t, n_v, dtype=torch.complex128, device="cuda")
        plan.correlator(U, D, C, S, stream=stream)
        torch.cuda.synchronize()
        site_recomputed = ctx.fp32_recomputed if fp32 else 0
        got = np.array([S[0, t, x].item() for t, x in pts])
        err = np.abs(got - ref) / np.abs(ref)
        accuracy = {"sites": len(pts), "rel_err_vs_oracle_max": float(err.max()),
                    "rel_err_vs_oracle_median": float(np.median(err)),
                    "rel_err_vs_oracle_q99": float(np.quantile(err, 0.99)),
                    "recomputed_with_site_values": site_recomputed,
                    "C_matches_C_only_call": bool(np.allclose(C.cpu().numpy(), C_main, rtol=1e-6, atol=0))}
        del S

    batched = None
    if headline and world == 1 and not args.no_batched:
        del U, D
        torch.cuda.empty_cache()
        batched = run_batched(local, stream, args.batched_sets)
        if "fp64" in compare:
            batched["vs_fp64_single_plan_he3"] = batched["value"] / compare["fp64"]["value"]

    if rank == 0:
        metric = METRIC if headline else f"sink-site contractions/sec ({args.op}, {Lb}^3x{Tb}, {args.algo}, {args.prec})"
        dtype = {"fp32": "f32", "mixed": "f32x2", "fp64": "f64"}[args.prec]
        config = {"workload": (f"{args.op}" + (" (stand-in for He-3 II)" if args.op == OPERATOR else "") +
                               f" {Lb}^3x{Tb}" + (f" ({n_t} slices)" if n_t != Tb else "") +
                               (f" ({n_v} sites/slice)" if n_v != Lb ** 3 else "") +
                               f", {n_sets} source(s) per GPU" +
                               (f", noise {args.noise}, kappa {args.kappa}" if args.noise else "")),
                  "algorithm": f"{args.algo} plan", "arithmetic": args.prec,
                  "sites_per_gpu": n_sites,
                  "l2": f"inputs {field_bytes / 1e9:.2f} GB per GPU" +
                        (", larger than L2" if field_bytes > 129e6 else ", smaller than L2"),
                  "canonical_terms": info["canonical_terms"], "index_size": info["index_size"]}
        if fp32:
            config["guard"] = {"site_threshold": guards[0], "slice_tolerance": guards[1],
                               "recomputed_sites_per_step": recomputed,
                               "recomputed_fraction": recomputed / max(1, n_sites)}
        if tuned:
            config["schedule"] = tuned
        line = {"metric": metric, "value": world * n_sites / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic (GPU-generated seeded recipe)",
                "config": config, "roofline": roofline, "compare": compare or None, "accuracy": accuracy,
                "batched": batched, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.destroy()
    ctx.close()


if __name__ == "__main__":
    main()
