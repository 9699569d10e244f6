"""Benchmark of the coupled multiphase LB step (MLUPS and HBM roofline).

Default workload: the 3-D Rayleigh-Taylor case, D3Q27 cumulant flow + phase
field, FP32 storage, 128 x 128 x 512 cells (8.4M), periodic in x and y,
half-way bounce-back walls in z, At 0.5, sqrt(g L) = 0.04, Re 1024, W 5,
M 0.02, with seeded velocity noise.  A step is one full coupled update of
every cell; its populations (3.6 GB) exceed L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank advances its own replica of the workload (the
update has no exchange between replicas); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

def _workloads():
    """the benchmark workloads: the shipped JSON case files of the package"""
    from paper_2101_06769_gb300 import cases
    return {name: cases.as_workload(cases.load(name)) for name in cases.shipped()}


WORKLOADS = _workloads()

# algorithmic bytes per cell update: every population read once and written
# once (phi is formed on chip and never stored by the fused kernels)
BYTES_PER_CELL = {3: 2 * (27 + 27) * 4, 2: 2 * (9 + 9) * 4}  # FP32
# shifted 16-bit storage: per population set one FP32 reference + (Q-1) codes
HBM_NOMINAL_GBS = 7900.0  # HBM3e nominal bandwidth of the part (context beside the measured peak)
BYTES_PER_CELL_16 = {3: 2 * 2 * (4 + 26 * 2), 2: 2 * 2 * (4 + 8 * 2)}
# reduced phase-field lattice (D3Q7 / D2Q5): f' and g read and written once,
# plus the stored previous phi u (D values) read and written once
BYTES_PER_CELL_RED = {3: 2 * 4 * (27 + 7 + 3), 2: 2 * 4 * (9 + 5 + 2)}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# of the step kernel, per cell, from the ncu capture summarised in profiles/;
# keyed by the SHA-256 of the kernel sources it was taken on, so that it is
# reported as null once those sources change.
TRAFFIC = {
    # 128x128x512 rt3d, one launch of step_fused3_kernel: 1891902208 B read + 1768638208 B written
    ("rt3d", "fp32"): {"bytes_per_cell": 3660540416 / 8388608, "sources": "b37d9ad5b72f47e6"},
    # same workload, step_fused3s_kernel<StoreF16>: 977621760 B read + 900893952 B written
    ("rt3d", "fp16"): {"bytes_per_cell": 1878515712 / 8388608, "sources": "b37d9ad5b72f47e6"},
    # same workload, reduced phase lattice (step_fused3_kernel, D3Q7 g): 1270872320 B read + 1197077760 B written
    ("rt3d", "reduced"): {"bytes_per_cell": 2467950080 / 8388608, "sources": "b37d9ad5b72f47e6"},
}
TRAFFIC_SOURCES = ["lbmp_common.cuh", "lbmp_tile.cuh", "lbmp_fused3_body.cuh", "lbmp_fused.cu", "lbmp_fused16.cu",
                   "lbmp_fused_r.cu"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2101_06769_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(workload, storage, cells):
    rec = TRAFFIC.get((workload, storage))
    if not rec or rec["sources"] != kernel_source_hash():
        return None
    return rec["bytes_per_cell"] * cells


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(local_ms, cells_per_rank, steps, dist=None):
    """Whole-job timing across ranks: the slowest rank's time counts (max over
    ranks) and the value is the cell updates of all ranks per second, in
    MLUPS.  Returns (max_ms, mlups)."""
    total_ms = float(local_ms)
    ws = 1
    if dist is not None and dist.is_initialized():
        import torch
        ws = dist.get_world_size()
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, ws * cells_per_rank * steps / (total_ms * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _oracle_rate(wl, depth, steps):
    """oracle MLUPS on a (nx, ny, depth) sub-box of the workload"""
    import oracle as O
    nx, ny = wl["dims"][0], wl["dims"][1]
    D = wl["D"]
    args = list(wl["args"])
    if wl["case"] == "rt":
        args[0] = depth / 2.0 if D == 3 else ny / 2.0
    dims = (nx, ny, depth) if D == 3 else (nx, ny, 1)
    o = O.Oracle(D, dims, wl["periodic"], **wl["phys"])
    o.init(wl["case"], args, seed=wl["seed"])
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = dims[0] * dims[1] * dims[2]
    return cells * steps / dt / 1e6, dims, dt


def cpu_baseline(wl, budget_s=12.0, max_state_gb=32.0):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of
    the workload: the full grid (when its FP64 state fits max_state_gb, else
    a horizontal slab of full x and y extent) with the workload's parameters,
    stepped on all cores for about budget_s seconds (at least one step), and
    one step on one thread beside it."""
    import oracle as O
    cores = O.get_threads()
    nx, ny, nz = wl["dims"]
    q = 27 if wl["D"] == 3 else 9
    per_plane_gb = 2 * 2 * q * 8 * nx * ny / 1e9  # two population sets of f' and g, FP64
    depth = nz if wl["D"] == 3 else 1
    if wl["D"] == 3 and depth * per_plane_gb > max_state_gb:
        depth = max(2, int(max_state_gb / per_plane_gb))
    what = "full grid" if depth == nz or wl["D"] == 2 else f"{nx}x{ny}x{depth} slab"
    rate, dims, dt = _oracle_rate(wl, depth, 1)
    steps = max(1, int(budget_s / max(dt, 1e-9)))
    if steps > 1:
        rate, dims, dt = _oracle_rate(wl, depth, steps)
    O.set_threads(1)
    try:
        rate1, _, dt1 = _oracle_rate(wl, depth, 1)
    finally:
        O.set_threads(cores)
    return {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{what} of the workload ({dims[0]}x{dims[1]}x{dims[2]}), {steps} steps on {cores} threads, "
                      f"FP64, {dt:.1f} s",
            "threads_1": {"value": rate1, "unit": "MLUPS", "cores": 1,
                          "sample": f"{what} of the workload, 1 step on 1 thread, FP64, {dt1:.1f} s"}}


def run_reference(args, wl):
    """The reference arm: the FP64 oracle on the host cores, one bounded
    sample of the workload per step, sized so that the whole run takes about
    two minutes."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    cores = O.get_threads()
    depth0 = 8 if wl["D"] == 3 else 1
    rate, dims, dt = _oracle_rate(wl, depth0, 1)
    per_sample = 120.0 / max(1, args.steps + args.warmup)
    cells_target = per_sample * rate * 1e6
    if wl["D"] == 3:
        depth = int(max(2, min(wl["dims"][2], cells_target // (wl["dims"][0] * wl["dims"][1]))))
    else:
        depth = 1
    vals, dts = [], []
    for k in range(args.warmup + args.steps):
        r, dims, dt = _oracle_rate(wl, depth, 1)
        if k >= args.warmup:
            vals.append(r)
            dts.append(dt)
    value = statistics.median(vals)
    cells = dims[0] * dims[1] * dims[2]
    sample = f"{dims[0]}x{dims[1]}x{dims[2]} slab of the workload, 1 step per timed step, FP64"
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(dts), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "grid": list(wl["dims"]),
                       "sample_cells": cells},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def kernel_name(args, D):
    if args.kernel == 1:
        return "phi_pass_kernel + step_simple_kernel"
    if args.storage != "fp32":
        return ("step_fused3s_kernel<Store%s>" if D == 3 else "step_fused2s_kernel<Store%s>") % args.storage.upper()
    if args.phase == "reduced":
        return "step_fused3_kernel (D3Q7 phase field)" if D == 3 else "step_fused2_kernel (D2Q5 phase field)"
    if D == 2:
        return "step_fused2_kernel"
    return "step_fused3b_kernel" if args.kernel == 2 else "step_fused3_kernel"


def time_steps(step, stream, n):
    """mean ms of one call of step() over n calls, CUDA events on the stream"""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(n):
        step()
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / n


# the batched form: one batch of uneven Rayleigh-Taylor members with sizes
# from the serving stream's ranges (3-D 64^3-128^3 cubes, 2-D 128^2-512^2
# squares), the same non-dimensional set-up scaled per member
BATCH_MIX = [(3, (64, 64, 64))] * 6 + [(3, (96, 96, 96))] * 4 + [(3, (128, 128, 128))] * 2 + \
            [(2, (128, 128, 1))] * 4 + [(2, (256, 256, 1))] * 4 + [(2, (512, 512, 1))] * 2
BATCH_MIX_DESC = ("6x64^3, 4x96^3, 2x128^3 D3Q27 + 4x128^2, 4x256^2, 2x512^2 D2Q9 Rayleigh-Taylor, FP32 "
                  "(sizes of the serving stream)")


def measure_batched(args, stream, peak, pg, n):
    """The batched form: one batch of the serving-size mix (BATCH_MIX), tuned
    and advanced by 16-step graph replays, next to the same members stepped
    one launch each.  Returns its record and the kernel launches it made."""
    from paper_2101_06769_gb300 import Batch, Domain
    doms, cells, byts, launches = [], 0, 0, 0
    b = Batch(stream=stream.cuda_stream)
    for k, (Dm, dims) in enumerate(BATCH_MIX):
        L = float(dims[0])
        per = (1, 1, 0) if Dm == 3 else (1, 0, 1)
        d = Domain(Dm, dims, per, stream=stream.cuda_stream, atwood=0.5, nu_ratio=1.0, Re=1024.0,
                   g_accel=0.04 ** 2 / L, L_ref=L, mobility=0.02, width=5.0)
        d.init("rt", [dims[Dm - 1] / 2.0, 0.1 * L, 1e-4, 1.0], seed=100 + k)
        b.add(d, 10 ** 6)
        doms.append(d)
        cells += d.N
        byts += BYTES_PER_CELL[Dm] * d.N
    if not args.no_autotune:
        b.autotune(reps=2)  # tile shape and planes per item of the batch kernels
    b.step(16)  # rebuild, capture and warm the graphs
    nb = 4 * max(1, n // 16)  # graph replays of 16 steps
    ms16 = time_steps(lambda: b.step(16), stream, nb)
    ms = ms16 / 16
    launches += nb * 16 * 3  # per step: 3-D batch kernel, 2-D batch kernel, epilogue
    _, mlups = aggregate(ms * nb * 16, cells, nb * 16, pg)
    gbs = byts / (ms * 1e-3) / 1e9
    res = {"mlups": mlups, "ms_per_step": ms, "members": len(doms), "cells": cells, "bytes_per_step": byts,
           "achieved_gbs": gbs, "frac": gbs / peak, "mix": BATCH_MIX_DESC, "steps": nb * 16}
    for d in doms:
        b.remove(d)
    b.close()
    # the same members stepped one domain at a time (one launch per member and
    # step, each with its own tuned launch shape): the plain one-domain form
    for d in doms:
        if not args.no_autotune:
            d.autotune(reps=2, cache=False)
    na = max(4, n // 4)

    def alone_round():
        for d in doms:
            d.step(1)

    ms_alone = time_steps(alone_round, stream, na)
    launches += na * len(doms)
    _, mlups_alone = aggregate(ms_alone * na, cells, na, pg)
    res["alone_mlups"] = mlups_alone
    res["alone_ms_per_step"] = ms_alone
    res["speedup_vs_alone"] = mlups / mlups_alone
    for d in doms:
        d.close()
    return res, launches


def measure_forms(args, wl, stream, peak, pg):
    """The other forms of the step on the same device: the workload with
    FP16 and BF16 shifted storage (fused kernel), and a batch of uneven
    domains advanced by the persistent batch kernels and CUDA graphs."""
    from paper_2101_06769_gb300 import Domain
    D = wl["D"]
    out, launches = {}, 0
    n = max(3, args.form_steps)
    for name in ("fp16", "bf16"):
        if name == args.storage or (D == 2 and args.kernel == 0):
            continue
        d = Domain(D, wl["dims"], wl["periodic"], stream=stream.cuda_stream, storage=STORAGE[name], **wl["phys"])
        d.init(wl["case"], wl["args"], seed=wl["seed"])
        if not args.no_autotune:
            d.autotune(reps=3, cache=False)
        d.step(5)
        ms = time_steps(lambda: d.step(1), stream, n)
        launches += n
        _, mlups = aggregate(ms * n, d.N, n, pg)
        bpc = BYTES_PER_CELL_16[D]
        gbs = bpc * d.N / (ms * 1e-3) / 1e9
        ob = d.observables()
        out[name] = {"mlups": mlups, "ms_per_step": ms, "bytes_per_cell": bpc, "achieved_gbs": gbs,
                     "frac": gbs / peak, "mass_drift_rel": ob.mass_drift_rel, "steps": n,
                     "traffic": traffic_per_launch(args.workload, name, d.N)}
        d.close()
    # the reduced phase-field lattice (D3Q7 / D2Q5 with the first-order
    # equilibrium and the correction term of Sec. 2.2) on the same workload
    if args.storage == "fp32" and args.kernel == 0 and args.phase == "full":
        from paper_2101_06769_gb300.lbmp import FLAG_PHASE_REDUCED
        phys = dict(wl["phys"])
        phys["flags"] = int(phys.get("flags", 0)) | FLAG_PHASE_REDUCED
        d = Domain(D, wl["dims"], wl["periodic"], stream=stream.cuda_stream, **phys)
        d.init(wl["case"], wl["args"], seed=wl["seed"])
        if not args.no_autotune:
            d.autotune(reps=3, cache=False)
        d.step(5)
        ms = time_steps(lambda: d.step(1), stream, n)
        launches += n
        _, mlups = aggregate(ms * n, d.N, n, pg)
        bpc = BYTES_PER_CELL_RED[D]
        gbs = bpc * d.N / (ms * 1e-3) / 1e9
        ob = d.observables()
        out["reduced_phase"] = {"mlups": mlups, "ms_per_step": ms, "bytes_per_cell": bpc, "achieved_gbs": gbs,
                                "frac": gbs / peak, "mass_drift_rel": ob.mass_drift_rel, "steps": n,
                                "kernel": "step_fused3_kernel (D3Q7 phase field)" if D == 3 else
                                "step_fused2_kernel (D2Q5 phase field)",
                                "traffic": traffic_per_launch(args.workload, "reduced", d.N)}
        d.close()
    # in-place AA storage (one population set each for f' and g, phi from a
    # pass of its own): half the state; the phi pass reads g once more and
    # writes phi (116 B/cell beyond the algorithmic 432), and the step reads it
    if args.storage == "fp32" and args.kernel == 0 and args.phase == "full" and D == 3:
        from paper_2101_06769_gb300.lbmp import FLAG_AA
        phys = dict(wl["phys"])
        phys["flags"] = int(phys.get("flags", 0)) | FLAG_AA
        d = Domain(D, wl["dims"], wl["periodic"], stream=stream.cuda_stream, **phys)
        d.init(wl["case"], wl["args"], seed=wl["seed"])
        d.step(4)
        ms = time_steps(lambda: d.step(1), stream, n)
        launches += 2 * n  # phi pass and step kernel
        _, mlups = aggregate(ms * n, d.N, n, pg)
        bpc = BYTES_PER_CELL[D]
        gbs = bpc * d.N / (ms * 1e-3) / 1e9
        ob = d.observables()
        out["aa_in_place"] = {"mlups": mlups, "ms_per_step": ms, "bytes_per_cell": bpc,
                              "overhead_bytes_per_cell": 27 * 4 + 8 + 8, "achieved_gbs": gbs, "frac": gbs / peak,
                              "state_bytes_per_cell": 2 * 27 * 4 + 8, "two_set_state_bytes_per_cell": 4 * 27 * 4,
                              "mass_drift_rel": ob.mass_drift_rel, "steps": n,
                              "kernel": "phi_pass_kernel + step_aa_kernel"}
        d.close()
    # batched form
    out["batched"], lb = measure_batched(args, stream, peak, pg, n)
    launches += lb
    mlups = out["batched"]["mlups"]
    out["serving"] = measure_serving(stream, mlups)
    # the same stream under a cap on the resident state: FP32 against 16-bit
    # storage of the D3Q27 requests (224 instead of 432 B/cell: more requests
    # resident), in a memory-bound regime (0.5 GB: the largest requests fit
    # only in 16-bit form) and a compute-bound one (2 GB)
    # capacity (requests served) and throughput are reported apart: under the
    # 0.5 GB cap FP32 cannot hold the largest requests at all, so the GLUPS of
    # the two forms are also compared on the requests whose FP32 state fits
    out["serving_budget"] = {}
    for gb in (0.5, 2.0):
        budget = int(gb * (1 << 30))
        rec = {"state_budget_bytes": budget,
               "fp32": measure_serving(stream, mlups, storage=0, state_budget=budget),
               "fp16": measure_serving(stream, mlups, storage=1, state_budget=budget)}
        rec["capacity"] = {"fp32_served": rec["fp32"]["done"], "fp16_served": rec["fp16"]["done"],
                           "requests": rec["fp32"]["requests"]}
        if rec["fp32"]["done"] < rec["fp32"]["requests"]:
            rec["same_requests"] = {
                "note": "only the requests whose FP32 state fits the cap, served by both forms",
                "fp32": measure_serving(stream, mlups, storage=0, state_budget=budget, fits=budget),
                "fp16": measure_serving(stream, mlups, storage=1, state_budget=budget, fits=budget)}
        out["serving_budget"]["%gGB" % gb] = rec
    out["_launches"] = launches
    return out


def measure_serving(stream, capacity_mlups, n=64, load=1.2, storage=0, state_budget=None, fits=None):
    """The serving loop (continuous batching) on the reduced serving stream:
    n seeded requests (RT or drop-on-sheet, 2-D 64^2-256^2 or 3-D
    64^3-128^3, We, Re and density ratio drawn as in the serving workload,
    200-2000 steps), Poisson arrivals at `load` times the capacity implied by
    the batched form's measured MLUPS.  fits: keep only the requests whose
    FP32 state is at most this many bytes (the same requests for every
    storage form)."""
    from paper_2101_06769_gb300 import serve
    kw = dict(sides2=(64, 128, 256), sides3=(64, 96, 128), steps_range=(200, 2000))
    probe = serve.request_stream(n, seed=7, **kw)
    work = sum(r.cells * r.steps for r in probe) / n
    rate = load * capacity_mlups * 1e6 / work
    reqs = serve.request_stream(n, seed=7, rate=rate, storage=storage, **kw)
    if fits is not None:  # FP32 state: two sets of f' and g, 4 bytes per population
        reqs = [r for r in reqs if 16 * (27 if r.D == 3 else 9) * r.cells <= fits]
    srv = serve.Server(stream=stream.cuda_stream, round_steps=64, state_budget=state_budget)
    peak = [0]
    admit = srv._admit

    def admit_and_count(r, now):
        admit(r, now)
        peak[0] = max(peak[0], len(srv.running))

    srv._admit = admit_and_count
    res = srv.run(reqs, max_wall=180.0)
    srv.close()
    res.update({"offered_load": load, "rate_rps": rate, "peak_resident": peak[0],
                "stream": "%d requests, seed 7, 2-D 64^2-256^2 / 3-D 64^3-128^3, 200-2000 steps, Poisson" % n})
    return res


def oracle_rates(wl, budget_s=8.0):
    """The FP64 oracle on 1 thread and on all host cores, each on a bounded
    slab of the workload (full x, y extent) for about budget_s seconds."""
    import oracle as O
    cores = O.get_threads()
    out = {}
    for nt in (1, cores):
        O.set_threads(nt)
        depth = min(wl["dims"][2], 4 if nt == 1 else 16) if wl["D"] == 3 else 1
        if wl["D"] == 3 and wl["dims"][0] * wl["dims"][1] > 400000:
            depth = 2
        rate, dims, dt = _oracle_rate(wl, depth, 1)
        steps = max(1, int(budget_s * rate * 1e6 / (dims[0] * dims[1] * dims[2])))
        rate, dims, dt = _oracle_rate(wl, depth, steps)
        out["threads_%d" % nt] = {"mlups": rate, "sample": "%dx%dx%d, %d steps, %.1f s" % (dims + (steps, dt))}
    O.set_threads(cores)
    out["cores"] = cores
    return out


def run_configs(args):
    """One JSON line per workload configuration of the benchmark set: MLUPS,
    algorithmic GB/s and roofline fraction per storage form, with the FP64
    oracle timed on 1 and on all host cores beside it."""
    import torch
    from paper_2101_06769_gb300 import Domain
    peak, _ = load_peaks()
    stream = torch.cuda.Stream()
    plan = [("rt2d", ["fp32"], 2000), ("rt3d", ["fp32", "fp16", "bf16"], 200),
            ("splash3d", ["fp32", "fp16", "bf16"], 100), ("splash3d_large", ["fp16", "fp32"], 30)]
    for name, forms, steps in plan:
        wl = WORKLOADS[name]
        D = wl["D"]
        line = {"config": name, "desc": wl["desc"], "grid": list(wl["dims"]), "forms": {}}
        for st in forms:
            d = Domain(D, wl["dims"], wl["periodic"], stream=stream.cuda_stream, storage=STORAGE[st], **wl["phys"])
            d.init(wl["case"], wl["args"], seed=wl["seed"])
            d.autotune(reps=2, cache=False)
            d.step(3)
            d.step(16)  # runs of 16 steps replay a captured graph (FP32): capture it before timing
            ms = time_steps(lambda: d.step(16), stream, max(1, steps // 16)) / 16
            bpc = BYTES_PER_CELL[D] if st == "fp32" else BYTES_PER_CELL_16[D]
            gbs = bpc * d.N / (ms * 1e-3) / 1e9
            ob = d.observables()
            line["forms"][st] = {"mlups": d.N / (ms * 1e-3) / 1e6, "ms_per_step": ms, "bytes_per_cell": bpc,
                                 "achieved_gbs": gbs, "frac": gbs / peak, "state_gb": 2 * d.state_bytes() / 1e9,
                                 "mass_drift_rel": ob.mass_drift_rel, "kinetic_energy": ob.kinetic_energy,
                                 "max_u": ob.max_u, "steps": steps + 3}
            d.close()
        if not args.no_cpu_baseline:
            line["oracle"] = oracle_rates(wl)
        print(json.dumps(line), flush=True)
    if args.serving_requests:
        from paper_2101_06769_gb300 import serve
        reqs = serve.request_stream(args.serving_requests, seed=7)
        work = sum(r.cells * r.steps for r in reqs) / len(reqs)
        cap = 8.5e9  # cell updates per second of the batched form (measured)
        rate = 1.2 * cap / work
        reqs = serve.request_stream(args.serving_requests, seed=7, rate=rate)
        srv = serve.Server(stream=stream.cuda_stream, round_steps=256)
        res = srv.run(reqs)
        srv.close()
        res.update({"config": "serving", "offered_load": 1.2, "rate_rps": rate,
                    "stream": "%d requests, seed 7, full serving ranges" % args.serving_requests})
        print(json.dumps(res), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rt3d", choices=sorted(WORKLOADS))
    ap.add_argument("--kernel", type=int, default=0,
                    help="0 fused (default), 1 reference pair, 2 fused with bulk-copy staging")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--grid", default=None, help="override nx,ny,nz (profiling on a smaller case)")
    ap.add_argument("--storage", default="fp32", choices=sorted(STORAGE))
    ap.add_argument("--phase", default="full", choices=["full", "reduced"],
                    help="phase-field lattice: the flow lattice, or D3Q7 / D2Q5 (FP32 only)")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16/BF16/batched form measurements")
    ap.add_argument("--batched-only", action="store_true",
                    help="measure the batched form alone (one JSON line), for profiling it")
    ap.add_argument("--form-steps", type=int, default=50)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--configs", action="store_true",
                    help="measure every workload configuration (one JSON line each) instead of the bench line")
    ap.add_argument("--serving-requests", type=int, default=0,
                    help="with --configs: also serve this many requests of the full serving stream")
    args = ap.parse_args()
    if args.phase == "reduced" and args.storage != "fp32":
        ap.error("the reduced phase lattice is stored in FP32 only")
    wl = dict(WORKLOADS[args.workload])
    if args.grid:
        dims = tuple(int(v) for v in args.grid.split(","))
        if wl["case"] == "rt":
            wl["args"] = [dims[wl["D"] - 1] / 2.0] + list(wl["args"][1:])
        wl["dims"] = dims
        wl["desc"] = wl["desc"] + f" (grid overridden to {dims[0]}x{dims[1]}x{dims[2]})"
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.configs:
        return run_configs(args)

    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("no CUDA device: the benchmark measures the GPU path only")
    torch.cuda.set_device(local)
    if args.batched_only:
        peak, _ = load_peaks()
        res, _ = measure_batched(args, torch.cuda.Stream(), peak, None, max(3, args.form_steps))
        print(json.dumps(dict(res, form="batched")), flush=True)
        return 0
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2101_06769_gb300 import Domain

    stream = torch.cuda.Stream()
    D = wl["D"]
    phys = dict(wl["phys"])
    if args.phase == "reduced":
        from paper_2101_06769_gb300.lbmp import FLAG_PHASE_REDUCED
        phys["flags"] = int(phys.get("flags", 0)) | FLAG_PHASE_REDUCED
    dom = Domain(D, wl["dims"], wl["periodic"], stream=stream.cuda_stream, storage=STORAGE[args.storage], **phys)
    dom.set_kernel(args.kernel)
    dom.init(wl["case"], wl["args"], seed=wl["seed"] + rank)
    cells = dom.N
    launch = {"chunk": 0, "ctas_per_sm": 0, "tuned": False}
    if not args.no_autotune and args.kernel != 1:
        # launch-shape autotuner of the library (trials do not advance the state)
        chunk, ctas, trials = dom.autotune(reps=3, cache=False)
        launch = {"chunk": chunk, "ctas_per_sm": ctas, "tuned": True, "trials": len(trials)}
    dom.step(args.warmup)
    dom.sync()

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    # timed region: K steps, each bracketed by events on the library's stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    time.sleep(0.3)
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        dom.step(1)
        ev[k][1].record(stream)
    t_end.record(stream)
    stream.synchronize()
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, mlups = aggregate(t_start.elapsed_time(t_end), cells, args.steps, pg)
    ms_per_step = total_ms / args.steps
    launches_per_step = 2 if args.kernel == 1 else 1

    # roofline of the step kernel: algorithmic bytes per launch / event time
    peak, peak_kind = load_peaks()
    kern_ms = statistics.mean(step_ms)
    bpc = BYTES_PER_CELL[D] if args.storage == "fp32" else BYTES_PER_CELL_16[D]
    form = args.storage
    if args.phase == "reduced":
        bpc, form = BYTES_PER_CELL_RED[D], "reduced"
    bytes_launch = bpc * cells
    achieved = bytes_launch / (kern_ms * 1e-3) / 1e9
    traffic = traffic_per_launch(args.workload, form, cells) if (args.kernel == 0 and not args.grid) else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "frac_nominal": achieved / HBM_NOMINAL_GBS, "traffic": traffic,
            "kernel": kernel_name(args, D),
            "bytes_per_cell": bpc}

    # end to end through the public API with host buffers: per step upload the
    # state from pinned host memory, advance one step, read the observables back
    nbytes = dom.state_bytes()
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    dom.download(host.data_ptr(), nbytes)
    dom.sync()
    e2e_steps = max(1, args.e2e_steps)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dom.upload(host.data_ptr(), nbytes)
        dom.step(1)
        dom.observables()
    torch.cuda.synchronize()
    e2e_ms, e2e_mlups = aggregate((time.perf_counter() - t0) * 1e3, cells, e2e_steps, pg)
    obs_bytes = 96 + 8 * 2 * (wl["dims"][D - 1])
    e2e = {"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": obs_bytes}

    ob = dom.observables()
    line = {"metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "grid": list(wl["dims"]), "cells": cells,
                       "storage": args.storage, "phase_lattice": args.phase, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas{ws}", "launch": launch},
            "roofline": roof, "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "health": ob.health, "mass_drift_rel": ob.mass_drift_rel}
    dom.close()
    if not args.no_forms and not args.grid:
        line["forms"] = measure_forms(args, wl, stream, peak, pg)
        line["gpu_launches_forms"] = line["forms"].pop("_launches")
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    if pg is not None:
        pg.barrier()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
