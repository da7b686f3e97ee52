#!/usr/bin/env python
"""Throughput of hybrid AB-/BA-GMRES on one GB300 (or N, one independent problem per GPU).

Workload (one "step"): the 512 x 512 fan-beam problem (720 views over 360 deg, 768 bins,
SID 1000, SDD 1500, 2 % Gaussian noise, seeded ellipse phantom), solved by hybrid AB-GMRES and
by hybrid BA-GMRES, 100 iterations each, lambda by the discrepancy principle (tau = 1.01).
The two solves of a step run as one batch (ct_batch: one CUDA graph whose two branches are
the solves, so the GPU runs them concurrently).
Metric: solver iterations per second over the whole job.  Inputs are resident in HBM when
the timed region starts; L2 is flushed (256 MiB write) between timed steps.

Reported beside the metric: per-phase device time and the roofline of the dominant kernel
(CUDA events on the launching stream, from a second timed region that runs the same solves one
after the other, so that every kernel's duration is its own) against ceilings measured in the
same run by the library's throughput probes (an L1 8-byte gather and a reciprocal + square
root pair), with the kernel's HBM fraction beside it; projector GUPS; an end-to-end number
through the C ABI with host buffers; the GPU clocks seen during the timed region; the FP64 CPU
oracle timed on a bounded sample of the same workload (with the GPU's error against it); and
"variants": the 16-bit Krylov bases at equal reconstruction error, the learned lambda rule, the
whole uneven 256-slice batch under one CUDA graph (default and autotuned launch shapes), the
matched pair and the 512^3 cone workload (FP32 and BF16 basis, with the error against the FP64
oracle on a reduced cone copy).

--workload slices times the 256-slice batch instead, split over the ranks by work (each rank
one captured graph of its slices; the whole batch is the fixed total, "scaling": "strong").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload fan512|slices]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hybrid GMRES iters/s + projector GUPS, % HBM roofline, at stated error vs FP64"
ITERS = 100
TAU = 1.01
L2_FLUSH_BYTES = 256 << 20
SM_COUNT = 152
# the kernels behind the phases the roofline is reported for, and their source files
PHASE_KERNELS = {"pixel_B": ("pixbp2d_kernel", "paper_2602_17892_gb300/csrc/proj2d.cu"),
                 "joseph_A": ("joseph2d_kernel", "paper_2602_17892_gb300/csrc/proj2d.cu"),
                 "arnoldi_cgs2": ("cgs_tile_kernel", "paper_2602_17892_gb300/csrc/arnoldi.cu")}
TRAFFIC_TABLE = os.path.join(ROOT, "profiles", "dram_traffic_fan512.md")


def kernel_traffic(name, shapes=None):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of the kernel behind `name` (for
    the pixel-driven B: the four-fold kernel when the launch shapes select it), from the
    committed ncu summary, or None when the kernel's source file has changed since the capture
    (its SHA-256 prefix no longer matches the one recorded beside the number)."""
    import hashlib
    kern, src = PHASE_KERNELS.get(name, (None, None))
    if name == "pixel_B" and shapes and shapes.get("b_views") == 4:
        kern = "pixbp2d_rot4_kernel"
    if kern is None or not os.path.exists(TRAFFIC_TABLE):
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
    for ln in open(TRAFFIC_TABLE):
        cells = [c.strip().strip("`") for c in ln.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == kern and cells[1] == src:
            return float(cells[3]) if cells[2] == sha else None
    return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


def measure_probe_peaks(torch, reps=1 << 16, trials=5):
    """Ceilings of the gather-bound projectors, measured now on this GPU with the library's
    throughput probes (CUDA events on the launching stream, best of `trials` one-wave launches
    of ~5-8 ms): 8-byte L1 gathers per second (each with its address arithmetic and one
    consuming FMA: the floor of one Joseph / pixel-driven sample) and reciprocal + square root
    pairs per second (the special-function work of one fan-beam pixel-driven sample)."""
    from paper_2602_17892_gb300 import _binding as Bn
    out = torch.empty(SM_COUNT * 16 * 256, device="cuda")
    st = torch.cuda.current_stream()
    res = {}
    for kind in ("gather8", "mufu"):
        Bn.ct_probe(kind, reps, out)
        torch.cuda.synchronize()
        best = None
        for _ in range(trials):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            ops = Bn.ct_probe(kind, reps, out)
            b.record(st)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        res[kind] = ops / (best * 1e-3) / 1e9          # G operations per second
    return res


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- ranks
def reduce_over_ranks(dist, device, total_ms, iters_done):
    """Whole-job numbers of the replicas (one independent problem per rank): the slowest
    rank's time and all ranks' iterations.  `dist` is None on one process."""
    if dist is None:
        return float(total_ms), float(iters_done)
    import torch
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    it = torch.tensor([float(iters_done)], device=device, dtype=torch.float64)
    dist.all_reduce(it, op=dist.ReduceOp.SUM)
    return float(t.item()), float(it.item())


# ----------------------------------------------------------------------------- workload
def workload(seed: int):
    import synth
    case = synth.fan512_case()
    return case["geom"], synth.ellipse_phantom(512, seed=case["phantom_seed"] + seed), case


def make_data_gpu(P, torch, G, geom, x_true, case, seed):
    """b = A x_true + e with the GPU projector (setup, untimed); e seeded, eta = 2 %."""
    import synth
    xt = torch.from_numpy(x_true.astype(np.float32).reshape(-1)).cuda()
    bt = torch.empty(G.m, device="cuda", dtype=torch.float32)
    P.ct_forward_A(G, xt, bt)
    torch.cuda.synchronize()
    b, e = synth.add_noise(bt.cpu().numpy().astype(np.float64), case["eta"], case["noise_seed"] + seed)
    b_dev = torch.from_numpy(b.astype(np.float32)).cuda()
    e_dev = torch.from_numpy(e.astype(np.float32)).cuda()
    be = torch.empty(G.n, device="cuda", dtype=torch.float32)
    P.ct_back_B(G, e_dev, be)
    torch.cuda.synchronize()
    return b, b_dev, float(np.linalg.norm(e)), float(torch.linalg.vector_norm(be.double()).item())


def run_step(P, G, b_dev, x_ab, x_ba, noise_ab, noise_ba):
    ia = P.ab_gmres_hybrid(G, b_dev, x_ab, max_iters=ITERS, rule="dp", noise_norm=noise_ab,
                           tau=TAU, history=False)
    ib = P.ba_gmres_hybrid(G, b_dev, x_ba, max_iters=ITERS, rule="dp", noise_norm=noise_ba,
                           tau=TAU, history=False)
    return ia["iters_done"] + ib["iters_done"]


def cpu_baseline(geom, b, noise_ab, noise_ba, P, torch, G, b_dev, iters=10):
    """FP64 oracle (as it stands) on a bounded sample: AB and BA, `iters` iterations each;
    the GPU's iterates at the same k are compared with it."""
    from oracle import proj as OP
    from oracle import solver as OS
    A, B = OP.operators(geom)
    t0 = time.perf_counter()
    ra = OS.hybrid_gmres("ab", A, B, b, iters, rule="dp", dp_target=TAU * noise_ab)
    rb = OS.hybrid_gmres("ba", A, B, b, iters, rule="dp", dp_target=TAU * noise_ba)
    dt = time.perf_counter() - t0
    xa = torch.zeros(G.n, device="cuda")
    xb = torch.zeros(G.n, device="cuda")
    P.ab_gmres_hybrid(G, b_dev, xa, max_iters=iters, rule="dp", noise_norm=noise_ab, tau=TAU,
                      history=False)
    P.ba_gmres_hybrid(G, b_dev, xb, max_iters=iters, rule="dp", noise_norm=noise_ba, tau=TAU,
                      history=False)
    torch.cuda.synchronize()
    err = lambda xg, xo: float(np.linalg.norm(xg.cpu().numpy() - xo) / np.linalg.norm(xo))
    return ({"value": 2 * iters / dt, "unit": "iters/s", "cores": OP.num_threads(),
             "kind": "oracle",
             "sample": f"hybrid AB and BA, {iters} iterations each, of the 512^2 fan workload "
                       f"(FP64, {dt:.1f} s)"},
            {"k": iters, "ab": err(xa, ra["x"]), "ba": err(xb, rb["x"]),
             "cone_reduced": cone_error_vs_fp64(P, torch)})


def cone_error_vs_fp64(P, torch, N=32, iters=ITERS):
    """The cone workload's error against the FP64 oracle, on a reduced copy (N^3, the recipe's
    views and detector scaled by N / 512, 1 % noise, hybrid AB-GMRES, K = 100, GCV): the GPU
    iterate with an FP32 and a BF16 basis against the oracle's iterate at the lambda the GPU's
    GCV chose (GCV is flat near its minimum; the 512^3 solve itself is beyond the oracle)."""
    import synth
    from oracle import proj as OP
    from oracle import solver as OS
    case = synth.cone512_case(N)
    g = case["geom"]
    x_true = synth.ellipsoid_phantom(N, seed=case["phantom_seed"], h=g.h)
    b, _ = synth.add_noise(OP.forward(g, x_true).reshape(-1), case["eta"], case["noise_seed"])
    b = b.astype(np.float32).astype(np.float64)
    G = P.Geom.from_geometry(g)
    b_dev = torch.from_numpy(b.astype(np.float32)).cuda()
    A, B = OP.operators(g)
    out = {"image": [N, N, N], "views": g.n_views, "detector": [g.n_det_v, g.n_det_u],
           "iters": iters, "rule": "gcv"}
    for basis in ("f32", "bf16"):
        x = torch.zeros(G.n, device="cuda")
        info = P.ab_gmres_hybrid(G, b_dev, x, max_iters=iters, rule="gcv", basis=basis)
        torch.cuda.synchronize()
        lam = float(info["lambdas"][iters - 1])
        ref = OS.hybrid_gmres("ab", A, B, b, iters, rule="fixed", lam_fixed=lam)["x"]
        xg = x.cpu().numpy().astype(np.float64)
        out[basis] = {"err_vs_fp64": float(np.linalg.norm(xg - ref) / np.linalg.norm(ref)),
                      "rre": OS.rre(xg, x_true), "lambda": lam}
    G.close()
    return out


# ----------------------------------------------------------------------------- ours
def bench_ours(args, rank, world, local_rank):
    import torch
    import paper_2602_17892_gb300 as P
    from paper_2602_17892_gb300 import _binding as Bn
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    geom, x_true, case = workload(rank)
    # one geometry object per problem of the batch (each owns its problem's workspace)
    G = P.Geom.from_geometry(geom)
    G_ba = P.Geom.from_geometry(geom)
    if args.launch_shapes:
        # fixed shapes (a profiler run repeats the shapes a plain run chose: the autotuner's
        # timings under a profiler would pick differently)
        fixed = dict(zip(SHAPE_KEYS, parse_shapes(args.launch_shapes)))
        for g in (G, G_ba):
            P.ct_geom_set_launch_shapes(g, fixed)
    batch = P.Batch([G, G_ba], ["ab", "ba"], max_iters=ITERS, rule="dp", tau=TAU,
                    autotune=not args.launch_shapes)
    shapes = P.ct_geom_get_launch_shapes(G)     # setup: projector launch shapes (autotuned)
    b, b_dev, noise_ab, noise_ba = make_data_gpu(P, torch, G, geom, x_true, case, rank)
    x_ab = torch.zeros(G.n, device="cuda")
    x_ba = torch.zeros(G.n, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()

    def batch_step():
        infos = batch.solve([b_dev, b_dev], [x_ab, x_ba], [noise_ab, noise_ba])
        return sum(i["iters_done"] for i in infos)

    for _ in range(args.warmup):
        batch_step()
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    iters_done = 0
    wall0 = time.perf_counter()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))            # L2 flush, outside the events
            evs[i][0].record(stream)
            iters_done += batch_step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = batch.launches() * args.steps
    step_ms = [a.elapsed_time(b_) for a, b_ in evs]
    total_ms = sum(step_ms)
    total_ms, iters_all = reduce_over_ranks(dist, "cuda", total_ms, iters_done)
    if dist:
        dist.barrier()
    value = iters_all / (total_ms / 1e3)

    # ---- per-kernel timing: the same two solves one after the other, per-phase CUDA events
    # on the launching stream (inside the batch's graph the two solves' kernels overlap)
    for _ in range(1):
        run_step(P, G, b_dev, x_ab, x_ba, noise_ab, noise_ba)
    torch.cuda.synchronize()
    seq_ms = 0.0
    Bn.ct_profile_enable(True)
    for i in range(args.steps):
        flush.fill_(float(i))
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        run_step(P, G, b_dev, x_ab, x_ba, noise_ab, noise_ba)
        eb.record(stream)
        torch.cuda.synchronize()
        seq_ms += ea.elapsed_time(eb)
    phases = Bn.ct_profile_collect()
    Bn.ct_profile_enable(False)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the region
    b_host = torch.from_numpy(b.astype(np.float32)).pin_memory()
    xa_host = torch.empty(G.n, dtype=torch.float32).pin_memory()
    xb_host = torch.empty(G.n, dtype=torch.float32).pin_memory()
    e2e_ms = 0.0
    e2e_iters = 0
    for i in range(args.steps):
        flush.fill_(float(i))
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        b_dev.copy_(b_host, non_blocking=True)
        e2e_iters += batch_step()
        xa_host.copy_(x_ab, non_blocking=True)
        xb_host.copy_(x_ba, non_blocking=True)
        eb.record(stream)
        torch.cuda.synchronize()
        e2e_ms += ea.elapsed_time(eb)
    e2e_ms, e2e_iters_all = reduce_over_ranks(dist, "cuda", e2e_ms, e2e_iters)
    e2e_value = e2e_iters_all / (e2e_ms / 1e3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- per-kernel rooflines against ceilings measured in this run
    peaks = _peaks()
    probe = measure_probe_peaks(torch)
    steps = args.steps
    f_ms, _, f_n = phases["forward_A"]          # groups = projector applications
    b_ms, _, b_n = phases["back_B"]
    a_ms, a_n, a_groups = phases["arnoldi"]
    # compulsory HBM bytes of one projector call: the input read once, the output written once
    proj_bytes = 4.0 * (G.n + G.m)
    kernels = {}
    if f_n:
        upd = G.a_samples * f_n
        gups = upd / (f_ms * 1e-3) / 1e9
        kernels["joseph_A"] = {"ms": f_ms, "launches": f_n, "gups": gups,
                               "peak_gups": probe["gather8"], "frac": gups / probe["gather8"],
                               "hbm_gbs": proj_bytes * f_n / (f_ms * 1e-3) / 1e9}
    if b_n:
        upd = G.b_samples * b_n
        gups = upd / (b_ms * 1e-3) / 1e9
        # fan: one tap-pair load per pixel-view pair and one rcp+sqrt (the four-fold kernel:
        # one rcp+sqrt per four pairs)
        rot4 = shapes.get("b_views") == 4
        pk = min(probe["gather8"], (4.0 if rot4 else 1.0) * probe["mufu"])
        kernels["pixel_B"] = {"ms": b_ms, "launches": b_n, "gups": gups, "peak_gups": pk,
                              "frac": gups / pk,
                              "hbm_gbs": proj_bytes * b_n / (b_ms * 1e-3) / 1e9}
    if a_groups:
        # algorithmic bytes of the Arnoldi steps of one AB and one BA solve (FP32 basis): CGS2
        # step k reads the k basis rows three times (dots; update fused with the second dots;
        # second update), reads q three times and writes q' and w_{k+1}: (3k + 5) L 4 bytes
        L_ab = geom.n_views * (geom.n_det_u + 4 + (-(geom.n_det_u + 4)) % 4)
        L_ba = geom.n + (-geom.n) % 4
        per_solve = lambda L: sum((3 * k + 5) * L * 4 for k in range(1, ITERS + 1))
        byts = (per_solve(L_ab) + per_solve(L_ba)) * steps
        gbs = byts / (a_ms * 1e-3) / 1e9
        kernels["arnoldi_cgs2"] = {"ms": a_ms, "launches": a_n, "gbs": gbs,
                                   "frac": gbs / peaks["hbm_gbs"]}
    for k in kernels.values():
        if "hbm_gbs" in k:
            k["hbm_frac"] = k["hbm_gbs"] / peaks["hbm_gbs"]
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    clk_sum = clk.summary()
    if dom == "arnoldi_cgs2":
        ach = kernels[dom]["gbs"]
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": kernel_traffic(dom),
                "peak_source": f"{peaks['source']} copy bandwidth (MEASURED_PEAKS.json)"}
    else:
        # gather/special-function bound projectors: their operands are L2-resident, so the
        # ceiling is the measured rate of the elementary work of one sample (probes above)
        kd = kernels[dom]
        src = ("ct_probe gather8 (one 8-byte L1 tap-pair load + one FMA per sample)"
               if kd["peak_gups"] == probe["gather8"] else
               "ct_probe mufu (one reciprocal + one square root per pixel-view pair)")
        roof = {"kernel": dom, "bound": "alu", "achieved": kd["gups"], "peak": kd["peak_gups"],
                "unit": "Gupdates/s", "frac": kd["frac"], "traffic": kernel_traffic(dom, shapes),
                "peak_source": f"measured in this run: {src}",
                "hbm": {"achieved_gbs": kd["hbm_gbs"], "peak_gbs": peaks["hbm_gbs"],
                        "frac": kd["hbm_frac"],
                        "bytes": "4 (n + m) per call: input read once, output written once"}}

    variants = None
    if world == 1 and args.variants != "none":
        variants = run_variants(P, torch, G, b_dev, x_true, noise_ab, args.variants)

    cpu = None
    err = None
    if world == 1 and not args.no_cpu_baseline:
        cpu, err = cpu_baseline(geom, b.astype(np.float32).astype(np.float64), noise_ab,
                                noise_ba, P, torch, G, b_dev)

    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipse phantom, b = A x + 2 % Gaussian noise)",
        "config": {"workload": "fan512: 512^2 fan-flat, 720 views/360 deg, 768 bins, "
                               "SID 1000, SDD 1500, 2 % noise; hybrid AB + BA, 100 its each, DP",
                   "image": [512, 512], "views": 720, "bins": 768, "iters_per_solve": ITERS,
                   "rule": "dp", "tau": TAU, "l2": "flushed between steps (256 MiB write)",
                   "execution": "the AB and BA solves as one ct_batch (one CUDA graph, two "
                                "concurrent branches)",
                   "launch_shapes": shapes,
                   "launch_shapes_from": "--launch-shapes" if args.launch_shapes else "autotuned",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "iters/s",
                "h2d_bytes_per_step": int(G.m * 4), "d2h_bytes_per_step": int(2 * G.n * 4)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": kernels,
        "phase_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
        "sequential_ms_per_step": seq_ms / args.steps,
        "per_kernel_timing": "second timed region: the same AB and BA solves one after the "
                             "other on one stream, CUDA events around every phase",
        "projector_gups": {k: v["gups"] for k, v in kernels.items() if "gups" in v},
        "err_vs_fp64": err,
        "clocks": clk_sum,
        "probe_peaks_gops": probe,
        "cpu_baseline": cpu,
        "variants": variants,
        "wall_s_timed": wall,
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- variants
# The forms the scope adds beside the plain FP32 method, each at its own workload, reported
# beside the main metric (rank 0, one GPU, after the timed region; not part of `value`).

def _timed(torch, fn, reps=1):
    """Device time (ms) of fn() on the current stream, CUDA events, after one warm-up call."""
    fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        out = fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, out


def variant_basis_precision(P, torch, G, b_dev, x_true, noise_ab, ks=tuple(range(10, 101, 10))):
    """Hybrid AB-GMRES on the 512^2 fan workload (DP) with the Krylov basis stored in FP32,
    FP16 and BF16, at equal reconstruction error: each basis solves with K = 10, 20, ..., 100;
    the target is the FP32 basis' error to the phantom at K = 100, and for each basis the first
    K that reaches it (within 0.1 %), its wall clock (device time of that solve) and the
    speed-up over the FP32 solve at K = 100 are reported, beside iterations/s and basis bytes."""
    xt = torch.from_numpy(x_true.astype(np.float32).reshape(-1)).cuda()
    nx = float(torch.linalg.vector_norm(xt))
    out, ref = {}, None
    L = G.m + (-G.m) % 4
    runs = {}
    for basis in ("f32", "f16", "bf16"):
        runs[basis] = {}
        for K in ks:
            x = torch.zeros(G.n, device="cuda")
            ms, _ = _timed(torch, lambda: P.ab_gmres_hybrid(G, b_dev, x, max_iters=K, rule="dp",
                                                            noise_norm=noise_ab, tau=TAU,
                                                            basis=basis, history=False))
            runs[basis][K] = (ms, float(torch.linalg.vector_norm(x - xt)) / nx)
            if K == ks[-1]:
                if ref is None:
                    ref = x.clone()
                out[basis] = {"iters_s": K / (ms * 1e-3), "ms_per_solve": ms,
                              "rre": runs[basis][K][1],
                              "rel_to_f32_basis": float(torch.linalg.vector_norm(x - ref) /
                                                        torch.linalg.vector_norm(ref)),
                              "basis_gb": (K + 1) * L * (4 if basis == "f32" else 2) / 1e9}
    target = runs["f32"][ks[-1]][1]
    t_ref = runs["f32"][ks[-1]][0]
    for basis in out:
        hit = next((K for K in ks if runs[basis][K][1] <= target * (1 + 1e-3)), None)
        out[basis]["rre_by_iters"] = {K: runs[basis][K][1] for K in ks}
        out[basis]["iters_to_f32_error"] = hit
        out[basis]["ms_to_f32_error"] = runs[basis][hit][0] if hit else None
        out[basis]["speedup_at_equal_error"] = t_ref / runs[basis][hit][0] if hit else None
    out["target_rre"] = target
    return out


def variant_matched(P, torch, G, b_dev, x_true, noise_ab):
    """The matched pair on the 512^2 fan workload: A^T alone (G samples/s, the same sample count
    as A) and hybrid AB-GMRES with B = A^T (LSQR's subspace, 100 its, DP) beside the unmatched
    solve: iterations/s and relative error to the phantom."""
    xt = torch.from_numpy(x_true.astype(np.float32).reshape(-1)).cuda()
    y = torch.rand(G.m, device="cuda")
    xo = torch.empty(G.n, device="cuda")
    ms_at, _ = _timed(torch, lambda: P.ct_back_AT(G, y, xo), reps=20)
    ms_b, _ = _timed(torch, lambda: P.ct_back_B(G, y, xo), reps=20)
    out = {"AT_ms": ms_at, "AT_gsamples_s": G.a_samples / (ms_at * 1e-3) / 1e9,
           "B_ms": ms_b}
    for kind in ("pixel", "adjoint"):
        P.ct_geom_set_backprojector(G, kind)
        x = torch.zeros(G.n, device="cuda")
        ms, _ = _timed(torch, lambda: P.ab_gmres_hybrid(G, b_dev, x, max_iters=ITERS, rule="dp",
                                                        noise_norm=noise_ab, tau=TAU,
                                                        history=False), reps=2)
        out[kind] = {"iters_s": ITERS / (ms * 1e-3), "ms_per_solve": ms,
                     "rre": float(torch.linalg.vector_norm(x - xt) / torch.linalg.vector_norm(xt))}
    P.ct_geom_set_backprojector(G, "pixel")
    return out


def slice_work(geom, iters):
    """Projector updates of one slice's solve (host estimate from the geometry: a Joseph A call
    samples about N points on each of n_views x n_det rays, a pixel-driven B call n_views x N^2
    pixel-view pairs), one A and one B per iteration."""
    N = max(geom.nx, geom.ny)
    return iters * geom.n_views * (geom.n_det_u * N + geom.nx * geom.ny)


def partition_slices(works, world):
    """Split slice indices over `world` ranks by work: largest first, each to the rank with the
    least work so far (ties to the lower rank).  Every slice lands on exactly one rank; the
    heaviest rank carries at most (total / world) + max(work).  Same answer on every rank (no
    communication)."""
    parts = [[] for _ in range(world)]
    load = [0] * world
    for i in sorted(range(len(works)), key=lambda j: (-works[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += works[i]
    return [sorted(p) for p in parts]


def _slice_problems(P, torch, cases):
    """Geometry, data b = A x_true + 1 % seeded noise (the library's own A) and a zero iterate
    for every slice."""
    import synth
    geoms, bs, xs = [], [], []
    for c in cases:
        g = c["geom"]
        G = P.Geom.from_geometry(g)
        x_true = synth.ellipse_phantom(g.nx, seed=c["phantom_seed"], ny=g.ny, h=g.h)
        xt = torch.from_numpy(x_true.astype(np.float32).reshape(-1)).cuda()
        bt = torch.empty(G.m, device="cuda")
        P.ct_forward_A(G, xt, bt)
        b, _ = synth.add_noise(bt.cpu().numpy().astype(np.float64), c["eta"], c["noise_seed"])
        geoms.append(G)
        bs.append(torch.from_numpy(b.astype(np.float32)).cuda())
        xs.append(torch.zeros(G.n, device="cuda"))
    return geoms, bs, xs


def variant_batched(P, torch, n_slices=256, iters=60):
    """The uneven batch (256 slices: N in {256..1024}, parallel/fan, 180-1440 views, 1 % noise,
    AB/BA by shape, 60 its, GCV): one graph replay of the whole batch with the geometries'
    default launch shapes (fresh geometries, no autotuning), then with autotuned shapes on the
    same geometries, then the same solves issued one after another; the per-kernel device time
    of those solves (events around every launch group) against the graph replay shows what the
    graph's concurrency and launch handling cost or save; device memory in use."""
    import synth
    from paper_2602_17892_gb300 import _binding as Bn
    cases = synth.batched_slices(256, seed=7)[:n_slices]
    geoms, bs, xs = _slice_problems(P, torch, cases)
    work = sum((G.a_samples + G.b_samples) * iters for G in geoms)
    total_iters = iters * len(cases)
    res = {"slices": len(cases), "iters_per_slice": iters,
           "pixels": int(sum(G.n for G in geoms)), "views_mean": float(np.mean(
               [c["geom"].n_views for c in cases]))}
    for tuned in (False, True):                 # default shapes first: autotuning rewrites them
        bt = P.Batch(geoms, ["auto"] * len(geoms), max_iters=iters, rule="gcv", autotune=tuned)
        shapes = {}
        for G in geoms:
            sh = P.ct_geom_get_launch_shapes(G)
            key = json.dumps(sh, sort_keys=True)
            shapes[key] = shapes.get(key, 0) + 1
        t0 = time.perf_counter()
        bt.solve(bs, xs)                          # first call captures the graph
        torch.cuda.synchronize()
        capture_s = time.perf_counter() - t0
        free, total = torch.cuda.mem_get_info()
        ms, _ = _timed(torch, lambda: bt.solve(bs, xs))
        key = "graph_tuned" if tuned else "graph_default_shapes"
        res[key] = {"iters_s": total_iters / (ms * 1e-3), "ms": ms,
                    "gups": work / (ms * 1e-3) / 1e9, "first_call_s": capture_s,
                    "launches_per_replay": bt.launches(), "device_gb_in_use": (total - free) / 1e9,
                    "launch_shapes_used": {k: v for k, v in shapes.items()}}
        bt.close()
    res["tuned_speedup_vs_default"] = res["graph_default_shapes"]["ms"] / res["graph_tuned"]["ms"]
    methods = ["ab" if G.m < G.n else "ba" for G in geoms]

    def sequential():
        for G, m, b, x in zip(geoms, methods, bs, xs):
            fn = P.ab_gmres_hybrid if m == "ab" else P.ba_gmres_hybrid
            fn(G, b, x, max_iters=iters, rule="gcv", history=False)
    ms, _ = _timed(torch, sequential)
    Bn.ct_profile_enable(True)
    sequential()
    torch.cuda.synchronize()
    ph = Bn.ct_profile_collect()
    Bn.ct_profile_enable(False)
    kern_ms = sum(v[0] for v in ph.values())
    res["sequential_solves"] = {"iters_s": total_iters / (ms * 1e-3), "ms": ms,
                                "gups": work / (ms * 1e-3) / 1e9,
                                "kernel_ms_sum": kern_ms,
                                "kernel_ms_by_phase": {k: v[0] for k, v in ph.items()}}
    res["graph_speedup_vs_sequential"] = res["sequential_solves"]["ms"] / res["graph_tuned"]["ms"]
    res["graph_ms_over_kernel_ms_sum"] = res["graph_tuned"]["ms"] / kern_ms
    for G in geoms:
        G.close()
    return res


def bench_slices(args, rank, world, local_rank, iters=60):
    """The 256-slice batch (N in {256..1024}, parallel/fan, 180-1440 views, 1 % noise, AB or BA
    by shape, 60 its, GCV) as the timed step.  The slices are split over the ranks by work
    (partition_slices, no communication); each rank captures its slices' solves as one CUDA
    graph (autotuned shapes) and replays it once per step.  value = all ranks' iterations /
    the slowest rank's time; the total work is fixed ("scaling": "strong")."""
    import torch
    import synth
    import paper_2602_17892_gb300 as P
    from paper_2602_17892_gb300 import _binding as Bn
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    cases = synth.batched_slices(256, seed=7)
    works = [slice_work(c["geom"], iters) for c in cases]
    mine = partition_slices(works, world)[rank]
    geoms, bs, xs = _slice_problems(P, torch, [cases[i] for i in mine])
    bt = P.Batch(geoms, ["auto"] * len(geoms), max_iters=iters, rule="gcv", autotune=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()
    step_iters = iters * len(geoms)
    for _ in range(args.warmup):
        bt.solve(bs, xs)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            bt.solve(bs, xs)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    total_ms, iters_all = reduce_over_ranks(dist, "cuda", total_ms, step_iters * args.steps)
    value = iters_all / (total_ms / 1e3)
    # end to end: this rank's data from pinned host memory and its iterates back, every step
    b_host = [b.cpu().pin_memory() for b in bs]
    x_host = [torch.empty(x.numel(), dtype=torch.float32).pin_memory() for x in xs]
    e2e_ms = 0.0
    for i in range(args.steps):
        flush.fill_(float(i))
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for bd, bh in zip(bs, b_host):
            bd.copy_(bh, non_blocking=True)
        bt.solve(bs, xs)
        for xh, xd in zip(x_host, xs):
            xh.copy_(xd, non_blocking=True)
        eb.record(stream)
        torch.cuda.synchronize()
        e2e_ms += ea.elapsed_time(eb)
    e2e_ms, e2e_iters = reduce_over_ranks(dist, "cuda", e2e_ms, step_iters * args.steps)
    h2d = sum(b.numel() * 4 for b in bs)
    d2h = sum(x.numel() * 4 for x in xs)
    # per-kernel device time: this rank's solves one after the other, events per launch group
    methods = ["ab" if G.m < G.n else "ba" for G in geoms]
    Bn.ct_profile_enable(True)
    for G, m, b, x in zip(geoms, methods, bs, xs):
        fn = P.ab_gmres_hybrid if m == "ab" else P.ba_gmres_hybrid
        fn(G, b, x, max_iters=iters, rule="gcv", history=False)
    torch.cuda.synchronize()
    ph = Bn.ct_profile_collect()
    Bn.ct_profile_enable(False)
    probe = measure_probe_peaks(torch)
    launches = bt.launches() * args.steps
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    a_upd = sum(G.a_samples for G in geoms) * iters
    b_upd = sum(G.b_samples for G in geoms) * iters
    kern = {"joseph_A": {"ms": ph["forward_A"][0], "gups": a_upd / (ph["forward_A"][0] * 1e-3) / 1e9,
                         "peak_gups": probe["gather8"]},
            "pixel_B": {"ms": ph["back_B"][0], "gups": b_upd / (ph["back_B"][0] * 1e-3) / 1e9,
                        "peak_gups": min(probe["gather8"], probe["mufu"])}}
    for k in kern.values():
        k["frac"] = k["gups"] / k["peak_gups"]
    dom = max(kern, key=lambda k: kern[k]["ms"])
    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipse phantoms, b = A x + 1 % Gaussian noise)",
        "config": {"workload": "slices256: 256 uneven slices, N in {256,512,768,1024}, "
                               "parallel/fan, 180-1440 views, 1 % noise; 60 its each, GCV, "
                               "AB or BA by shape",
                   "slices_this_rank": len(geoms), "l2": "flushed between steps (256 MiB write)",
                   "execution": "each rank: its slices' solves as one CUDA graph (concurrent "
                                "branches, autotuned launch shapes)",
                   "parallelism": f"slices split by work over {world} rank(s)"},
        "e2e": {"value": e2e_iters / (e2e_ms / 1e3), "unit": "iters/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": {"kernel": dom, "bound": "alu", "achieved": kern[dom]["gups"],
                     "peak": kern[dom]["peak_gups"], "unit": "Gupdates/s",
                     "frac": kern[dom]["frac"], "traffic": None,
                     "peak_source": "measured in this run: ct_probe gather8 / mufu"},
        "kernels": kern,
        "phase_ms_sequential": {k: v[0] for k, v in ph.items()},
        "clocks": clk.summary(),
        "probe_peaks_gops": probe,
        "cpu_baseline": None,
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def variant_cone(P, torch, iters=ITERS):
    """The 512^3 cone workload (400 views, 768 x 768 detector, 1 % noise), hybrid AB-GMRES,
    GCV, with the Krylov basis in FP32 and in BF16: iterations/s, projector GUPS, basis bytes,
    relative error to the phantom and between the two."""
    import synth
    from paper_2602_17892_gb300 import _binding as Bn
    case = synth.cone512_case()
    g = case["geom"]
    x_true = synth.ellipsoid_phantom(g.nx, seed=case["phantom_seed"], h=g.h)
    G = P.Geom.from_geometry(g)
    shapes = P.ct_geom_autotune(G)
    xt = torch.from_numpy(x_true.astype(np.float32).reshape(-1)).cuda()
    del x_true
    bt = torch.empty(G.m, device="cuda")
    P.ct_forward_A(G, xt, bt)
    b, _ = synth.add_noise(bt.cpu().numpy().astype(np.float64), case["eta"], case["noise_seed"])
    b_dev = torch.from_numpy(b.astype(np.float32)).cuda()
    del b, bt
    out = {"image": [g.nx, g.ny, g.nz], "views": g.n_views, "detector": [g.n_det_v, g.n_det_u],
           "iters": iters, "rule": "gcv", "launch_shapes": shapes}
    ref = None
    for basis in ("bf16", "f32"):
        x = torch.zeros(G.n, device="cuda")
        P.ab_gmres_hybrid(G, b_dev, x, max_iters=2, rule="gcv", basis=basis, history=False)
        torch.cuda.synchronize()
        Bn.ct_profile_enable(True)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        P.ab_gmres_hybrid(G, b_dev, x, max_iters=iters, rule="gcv", basis=basis, history=False)
        e1.record(st)
        torch.cuda.synchronize()
        ph = Bn.ct_profile_collect()
        Bn.ct_profile_enable(False)
        ms = e0.elapsed_time(e1)
        L = G.m  # padded sinogram entries are reported by the library's own basis size below
        out[basis] = {"iters_s": iters / (ms * 1e-3), "s_per_solve": ms / 1e3,
                      "rre": float(torch.linalg.vector_norm(x - xt) / torch.linalg.vector_norm(xt)),
                      "phase_ms": {k: v[0] for k, v in ph.items()},
                      "gups_A": G.a_samples * ph["forward_A"][2] / (ph["forward_A"][0] * 1e-3) / 1e9,
                      "gups_B": G.b_samples * ph["back_B"][2] / (ph["back_B"][0] * 1e-3) / 1e9,
                      "basis_gb_approx": (iters + 1) * L * (2 if basis == "bf16" else 4) / 1e9,
                      "max_mem_gb": torch.cuda.max_memory_allocated() / 1e9}
        if ref is None:
            ref = x.clone()
        else:
            out["rel_bf16_vs_f32"] = float(torch.linalg.vector_norm(ref - x) /
                                           torch.linalg.vector_norm(x))
        del x
    G.close()
    return out


def variant_learned(P, torch, n_test=16, K=30):
    """The learned lambda rule (network trained by the library on 20 000 solves of the
    256^2 parallel recipe) against GCV and DP on held-out problems: mean relative error,
    device time per solve, and the iteration count at which the learned rule first matches
    GCV's error at K."""
    from paper_2602_17892_gb300 import lambda_net as LN
    net, meta = LN.load_params()
    geom = LN.training_geometry()
    G = P.Geom.from_geometry(geom)
    res = {"rre": {"learned": [], "gcv": [], "dp": []}, "ms_per_solve": {}, "iters_to_gcv_error": []}
    times = {"learned": 0.0, "gcv": 0.0, "dp": 0.0}
    x = torch.zeros(G.n, device="cuda")
    for sd in range(30_000_000, 30_000_000 + n_test):
        xt, b, nn = LN.make_problem(geom, G, sd)
        nx = float(torch.linalg.vector_norm(xt))
        for rule in ("learned", "gcv", "dp"):
            ms, _ = _timed(torch, lambda: P.ab_gmres_hybrid(
                G, b, x, max_iters=K, rule=rule, noise_norm=nn, tau=TAU, history=False,
                lambda_net=net if rule == "learned" else None))
            times[rule] += ms
            res["rre"][rule].append(float(torch.linalg.vector_norm(x - xt)) / nx)
        target = res["rre"]["gcv"][-1]
        k_hit = None
        for k in range(5, K + 1, 5):
            P.ab_gmres_hybrid(G, b, x, max_iters=k, rule="learned", history=False, lambda_net=net)
            if float(torch.linalg.vector_norm(x - xt)) / nx <= target:
                k_hit = k
                break
        res["iters_to_gcv_error"].append(k_hit)
    G.close()
    res["mean_rre"] = {k: float(np.mean(v)) for k, v in res["rre"].items()}
    res["ms_per_solve"] = {k: v / n_test for k, v in times.items()}
    res["K"] = K
    res["train_solves"] = meta.get("train_solves")
    lr, gr = np.array(res["rre"]["learned"]), np.array(res["rre"]["gcv"])
    res["per_problem_rre"] = {"learned": [float(v) for v in lr], "gcv": [float(v) for v in gr],
                              "dp": [float(v) for v in res["rre"]["dp"]]}
    res["problems_within_1pct_of_gcv"] = int(np.sum(lr <= gr * 1.01))
    res["problems_better_than_gcv"] = int(np.sum(lr < gr))
    res["n_test"] = n_test
    del res["rre"]
    return res


def run_variants(P, torch, G, b_dev, x_true, noise_ab, which):
    out = {}
    jobs = {"basis_precision_fan512_ab": lambda: variant_basis_precision(P, torch, G, b_dev, x_true, noise_ab),
            "learned_lambda_parallel256": lambda: variant_learned(P, torch),
            "batched_slices_256": lambda: variant_batched(P, torch),
            "matched_pair_fan512_ab": lambda: variant_matched(P, torch, G, b_dev, x_true, noise_ab),
            "cone512": lambda: variant_cone(P, torch)}
    for name, fn in jobs.items():
        if which != "all" and name not in which.split(","):
            continue
        try:
            t0 = time.perf_counter()
            out[name] = fn()
            out[name]["wall_s"] = time.perf_counter() - t0
        except Exception as exc:                 # reported, never hides the main metric
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- projectors only
def bench_projectors(args):
    """A and B alone on one workload (fan512, cone256 or cone512): device time per call with
    CUDA events, GUPS; the command the projector profiles in profiles/ are taken with."""
    import torch
    import synth
    import paper_2602_17892_gb300 as P
    if args.projectors == "fan512":
        g = synth.fan512_case()["geom"]
        x = synth.ellipse_phantom(512, seed=0)
    else:
        N = 256 if args.projectors == "cone256" else 512
        g = synth.cone512_case(N)["geom"]
        x = synth.ellipsoid_phantom(N, seed=0)
    G = P.Geom.from_geometry(g)
    if args.launch_shapes:
        shapes = dict(zip(SHAPE_KEYS, parse_shapes(args.launch_shapes)))
        P.ct_geom_set_launch_shapes(G, shapes)
    else:
        shapes = P.ct_geom_autotune(G) if not args.no_autotune else None
    xd = torch.from_numpy(x.astype(np.float32).reshape(-1)).cuda()
    yd = torch.empty(G.m, device="cuda")
    xb = torch.empty(G.n, device="cuda")
    for _ in range(args.warmup):
        P.ct_forward_A(G, xd, yd)
        P.ct_back_B(G, yd, xb)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(st)
    for _ in range(args.steps):
        P.ct_forward_A(G, xd, yd)
    ev[1].record(st)
    for _ in range(args.steps):
        P.ct_back_B(G, yd, xb)
    ev[2].record(st)
    torch.cuda.synchronize()
    a_ms = ev[0].elapsed_time(ev[1]) / args.steps
    b_ms = ev[1].elapsed_time(ev[2]) / args.steps
    print(json.dumps({"projectors": args.projectors, "image": list(g.image_shape), "views": g.n_views,
                      "detector": [g.n_det_v, g.n_det_u], "launch_shapes": shapes,
                      "A_ms": a_ms, "B_ms": b_ms, "A_gups": G.a_samples / (a_ms * 1e-3) / 1e9,
                      "B_gups": G.b_samples / (b_ms * 1e-3) / 1e9, "steps": args.steps,
                      "warmup": args.warmup}), flush=True)


# ----------------------------------------------------------------------------- reference arm
def bench_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores: each step is a bounded sample of the workload
    (hybrid AB and BA, a few iterations each)."""
    if rank != 0:
        return
    import synth
    from oracle import proj as OP
    from oracle import solver as OS
    geom, x_true, case = workload(0)
    b, e = synth.add_noise(OP.forward(geom, x_true).reshape(-1), case["eta"], case["noise_seed"])
    b = b.astype(np.float32).astype(np.float64)
    A, B = OP.operators(geom)
    nab, nba = float(np.linalg.norm(e)), float(np.linalg.norm(B(e)))
    its = 4

    def step():
        OS.hybrid_gmres("ab", A, B, b, its, rule="dp", dp_target=TAU * nab)
        OS.hybrid_gmres("ba", A, B, b, its, rule="dp", dp_target=TAU * nba)
        return 2 * its

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    n = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    value = n / dt
    sample = f"hybrid AB and BA, {its} iterations each, of the 512^2 fan workload, per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded ellipse phantom)",
        "config": {"workload": "fan512: 512^2 fan-flat, 720 views/360 deg, 768 bins, "
                               "SID 1000, SDD 1500, 2 % noise; hybrid AB + BA, DP"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": OP.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def check_ranks(gpus, env):
    """The launch must match --gpus: one process per GPU, started by torchrun (WORLD_SIZE).
    Returns an error message, or None when the launch is consistent."""
    world = int(env.get("WORLD_SIZE", 1))
    if gpus < 1:
        return "--gpus must be >= 1"
    if "WORLD_SIZE" not in env and gpus > 1:
        return (f"--gpus {gpus} needs one process per GPU: launch with python -m "
                f"torch.distributed.run --nproc-per-node {gpus} --master-addr 127.0.0.1 "
                f"bench.py --gpus {gpus}")
    if world != gpus:
        return f"--gpus {gpus} does not match WORLD_SIZE={world}"
    return None


SHAPE_KEYS = ("a_threads", "a_views", "a_slab", "b_rows", "b_views", "a_rays", "a_warp_views",
              "b_warp_rows")


def parse_shapes(text):
    """Six or eight integers in SHAPE_KEYS order (six: one view per Joseph warp, one pixel row
    per B warp)."""
    vals = [int(v) for v in text.split(",")]
    if len(vals) == 6:
        vals += [1, 1]
    if len(vals) != len(SHAPE_KEYS):
        raise SystemExit("--launch-shapes takes six or eight integers: " + ",".join(SHAPE_KEYS))
    return vals


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["fan512", "slices"], default="fan512")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--projectors", choices=["fan512", "cone256", "cone512"], default=None,
                    help="time A and B alone on this workload instead of the solver benchmark")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch-shapes", default=None,
                    help="fixed projector launch shapes (solver and projector benchmarks) "
                         "instead of autotuning: " + ",".join(SHAPE_KEYS) + " as six or eight integers")
    ap.add_argument("--variants", default="all",
                    help="'all', 'none' or a comma list of: basis_precision_fan512_ab, "
                         "learned_lambda_parallel256, batched_slices_256, cone512, "
                         "matched_pair_fan512_ab")
    args = ap.parse_args()
    msg = check_ranks(args.gpus, os.environ)
    if msg:
        print(f"bench.py: {msg}", file=sys.stderr)
        sys.exit(2)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        from oracle import proj as OP
        OP.build_oracle()
        bench_reference(args, rank, world)
        return
    from paper_2602_17892_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    else:                       # the other ranks wait for rank 0's build
        t0 = time.time()
        while B.needs_build() and time.time() - t0 < 600:
            time.sleep(1.0)
    if args.projectors:
        bench_projectors(args)
        return
    if args.workload == "slices":
        bench_slices(args, rank, world, local_rank)
        return
    from oracle import proj as OP
    OP.build_oracle()
    bench_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
