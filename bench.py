"""Benchmark: docking evaluations per second on a 128^3 lattice.

One step = one registration through the whole path on resident inputs: the
global Super-Fibonacci search, the local GeoBall-SF search around its best
orientation, top-K, and the refinement of the K candidates (the object grid
and its spectrum are built once per object, before the timed region, and timed
separately; the end-to-end figure rebuilds them every step from host arrays).

Prints one JSON line (rank 0).  Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs its own registration (independent problems,
weak scaling); the timed region is bracketed by barriers and the slowest
rank's time is used.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "large128"
N_GLOBAL = 32768
N_LOCAL = 5000            # min(5000, n_rot / 4) local GeoBall-SF samples
THETA = math.radians(5.0)
TOP_K = 64
METRIC = "docking evals/s @128^3"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


SERVE_SIZES = (32, 64, 96, 128)


def serving_mix(synth, n_req=24, seed=11):
    """Uneven requests shaped like the batched workload: lattice side uniform
    over {32, 64, 96, 128} at h = 16 mm / N, trajectories of 100-2000 poses,
    probe radius 0.5-1.5 mm (length 12 mm), 1000-4000 global SF rotations plus
    a quarter as many local ones, top-8 refined; 8 objects (two per side),
    each with its own trajectory, shared by the requests."""
    rng = np.random.default_rng(seed)
    works = []
    for k, N in enumerate(SERVE_SIZES * 2):
        works.append(synth.make_workload("free64", replicate=100 + k, N=N, h=16.0 / N, n_theta=48, n_phi=96,
                                         poses=int(rng.integers(100, 2001)), radius=float(rng.uniform(0.5, 1.5)),
                                         noncontact=0.0, noise_t=0.02, noise_r=0.0, lines=3, pitch=1.5))
    reqs = []
    for _ in range(n_req):
        wi = int(rng.integers(0, len(works)))
        ng = int(rng.integers(1000, 4001))
        reqs.append((wi, ng, ng // 4))
    return works, reqs


def cufft_comparison(ctx, ob, sw, w, stream, n_rot=16, batch=8):
    """The correlation of the search done with cuFFT (through torch.fft) for
    comparison only: S_R from the library's voxeliser (bit-identical), then
    R2C, the product with conj(F(O)), C2R and the argmax over the M^3 canvas,
    batch rotations at a time.  Returns the cuFFT device time per rotation
    (CUDA events; the voxeliser excluded, as in the kernels it is set against)
    and the largest score difference to the library's peaks."""
    import torch
    N, M = w.N, 2 * w.N
    quats = synth_rotations(n_rot)
    bits, _ = sw.voxelise(quats)
    G, _ = ob.export_grid()
    with torch.cuda.stream(stream):
        Og = torch.zeros((M, M, M), dtype=torch.float32, device="cuda")
        Og[:N, :N, :N] = torch.from_numpy(G).cuda()
        FOc = torch.conj(torch.fft.rfftn(Og))
        del Og
        Sd = torch.from_numpy(bits).cuda()
        best = torch.empty(n_rot, dtype=torch.float32, device="cuda")

        def run():
            for b0 in range(0, n_rot, batch):
                Sp = torch.zeros((batch, M, M, M), dtype=torch.float32, device="cuda")
                Sp[:, :N, :N, :N] = Sd[b0:b0 + batch].float()
                C = torch.fft.irfftn(torch.fft.rfftn(Sp, dim=(1, 2, 3)) * FOc, s=(M, M, M), dim=(1, 2, 3))
                best[b0:b0 + batch] = C.reshape(batch, -1).max(dim=1).values
        run()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        run()
        ev1.record(stream)
    ev1.synchronize()
    us = ev0.elapsed_time(ev1) * 1000.0 / n_rot
    _, pk = ctx.search_so3(ob, sw, n_rot, 1, sampler=3, quats=quats, want_peaks=True)
    diff = float(np.max(np.abs(best.cpu().numpy() - pk["score"])))
    torch.cuda.empty_cache()
    return {"us_per_rotation": round(us, 1), "rotations": n_rot, "batch": batch,
            "path": "torch.fft (cuFFT) R2C + conj(F(O)) product + C2R + argmax, S_R from the library's voxeliser",
            "max_peak_score_diff": round(diff, 4)}


def config4_mix(synth, n_req, n_obj=16, seed=41):
    """Requests shaped like the batched-instances workload: lattice side
    uniform over {32, 64, 96, 128} at h = 16 mm / N, trajectories of U[100,
    5000] poses, probe radius U[0.5, 1.5] mm (length 12 mm), U[1000, 16000]
    orientation samples (80 % global SF, 20 % local GeoBall-SF), top-8
    refined; n_obj objects (a quarter per side), each with its own
    trajectory, shared by the requests."""
    rng = np.random.default_rng(seed)
    works = []
    for k in range(n_obj):
        N = SERVE_SIZES[k % 4]
        works.append(synth.make_workload("free64", replicate=200 + k, N=N, h=16.0 / N, n_theta=48, n_phi=96,
                                         poses=int(rng.integers(100, 5001)), radius=float(rng.uniform(0.5, 1.5)),
                                         noncontact=0.0, noise_t=0.02, noise_r=0.0, lines=3, pitch=1.5))
    reqs = []
    for _ in range(n_req):
        n = int(rng.integers(1000, 16001))
        reqs.append((int(rng.integers(0, n_obj)), int(0.8 * n), n - int(0.8 * n)))
    return works, reqs


def batch_study(ctx, synth, n_req):
    """dock_register_batch on the mix against the plain loop of dock_register
    (one request at a time), same requests, results compared bit for bit."""
    works, reqs = config4_mix(synth, n_req)
    handles = [(ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N),
                ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)) for w in works]
    req_t = [(handles[i][0], handles[i][1], ng, nl, THETA, 8) for i, ng, nl in reqs]
    try:
        for N in SERVE_SIZES:   # warm every lattice side
            i = next(k for k, w in enumerate(works) if w.N == N)
            ctx.register(handles[i][0], handles[i][1], 256, 64, THETA, 8)
        t0 = time.perf_counter()
        plain = [ctx.register(*r) for r in req_t]
        t_plain = time.perf_counter() - t0
        t0 = time.perf_counter()
        batch = ctx.register_batch(req_t)
        t_batch = time.perf_counter() - t0
        same = all(np.array_equal(a["q"], b["q"]) and np.array_equal(a["t"], b["t"]) and a["J"] == b["J"]
                   for a, b in zip(plain, batch))
        evals = sum(ng + nl for _, ng, nl in reqs)
        return {"requests": len(reqs), "objects": len(works), "evals": evals,
                "mix": "N uniform over {32,64,96,128} at 16/N mm, 100-5000 poses, r 0.5-1.5 mm, 1000-16000 "
                       "samples (80% SF + 20% GeoBall-SF), top-8",
                "plain_regs_per_s": round(len(reqs) / t_plain, 3), "batch_regs_per_s": round(len(reqs) / t_batch, 3),
                "batch_vs_plain": round(t_plain / t_batch, 3), "plain_s": round(t_plain, 2),
                "batch_s": round(t_batch, 2), "results_equal_plain": bool(same)}
    finally:
        for ob, sw in handles:
            ob.close()
            sw.close()


def serving_study(ctx, synth, n_req, rates):
    """Poisson arrivals of n_req requests of the serving mix at each rate
    (req/s): served regs/s and p50/p99/p99.9 latency (submission to result),
    every result compared with the request registered alone."""
    works, reqs = serving_mix(synth, n_req=n_req)
    handles = [(ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N),
                ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)) for w in works]
    req_t = [(handles[wi][0], handles[wi][1], ng, nl, THETA, 8) for wi, ng, nl in reqs]
    out = []
    try:
        ctx.register(*req_t[0])
        n_plain = min(40, n_req)
        t0 = time.perf_counter()
        alone = [ctx.register(*r) for r in req_t[:n_plain]]
        t_plain = time.perf_counter() - t0
        for rate in rates:
            gaps = np.random.default_rng(int(rate * 100)).exponential(1.0 / rate, size=n_req)
            arrivals = np.cumsum(gaps) - gaps[0]
            tickets, done = {}, {}
            t0 = time.perf_counter()
            nxt = 0
            while len(done) < n_req:
                now = time.perf_counter() - t0
                while nxt < n_req and arrivals[nxt] <= now:
                    tickets[ctx.submit(req_t[nxt])] = nxt
                    nxt += 1
                for t, i in list(tickets.items()):
                    r = ctx.poll(t, timeout_us=0)
                    if r is not None:
                        done[i] = r
                        del tickets[t]
                time.sleep(0.0005)
            span = time.perf_counter() - t0
            lat = np.array([done[i]["latency_ms"] for i in range(n_req)])
            same = all(np.array_equal(done[i]["q"], alone[i]["q"]) and done[i]["J"] == alone[i]["J"]
                       for i in range(n_plain))
            out.append({"rate_per_s": rate, "requests": n_req, "served_regs_per_s": round(n_req / span, 3),
                        "p50_ms": round(float(np.percentile(lat, 50)), 1),
                        "p99_ms": round(float(np.percentile(lat, 99)), 1),
                        "p999_ms": round(float(np.percentile(lat, 99.9)), 1),
                        "results_equal_alone": bool(same)})
        return {"mix": "N uniform over {32,64,96,128}, 100-2000 poses, r 0.5-1.5 mm, 1000-4000 + 25% rotations, "
                       "top-8, 8 objects", "plain_regs_per_s": round(n_plain / t_plain, 3), "rates": out}
    finally:
        for ob, sw in handles:
            ob.close()
            sw.close()


def synth_rotations(n, seed=5):
    from paper_2605_21398_gb300 import synth
    return synth.random_unit_quats(n, seed)


def serving_experiment(ctx, synth):
    """Plain loop (dock_register one request at a time) against the serving
    engine (dock_submit/dock_poll): a burst of all requests for throughput,
    then Poisson arrivals at 80 % of the burst rate for latency."""
    works, reqs = serving_mix(synth)
    handles = [(ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N),
                ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)) for w in works]
    req_t = [(handles[wi][0], handles[wi][1], ng, nl, THETA, 8) for wi, ng, nl in reqs]
    try:
        ctx.register(*req_t[0])                      # warm-up of every code path
        t0 = time.perf_counter()
        plain = [ctx.register(*r) for r in req_t]
        t_plain = time.perf_counter() - t0

        def serve(arrivals):
            tickets, done = {}, {}
            t0 = time.perf_counter()
            nxt = 0
            while len(done) < len(req_t):
                now = time.perf_counter() - t0
                while nxt < len(req_t) and arrivals[nxt] <= now:
                    tickets[ctx.submit(req_t[nxt])] = nxt
                    nxt += 1
                for t, i in list(tickets.items()):
                    r = ctx.poll(t, timeout_us=0)
                    if r is not None:
                        done[i] = r
                        del tickets[t]
                time.sleep(0.0005)
            return [done[i] for i in range(len(req_t))], time.perf_counter() - t0

        burst, t_burst = serve([0.0] * len(req_t))
        rate = 0.8 * len(req_t) / t_burst
        gaps = np.random.default_rng(5).exponential(1.0 / rate, size=len(req_t))
        poisson, t_pois = serve(list(np.cumsum(gaps) - gaps[0]))
        same = all(np.array_equal(a["q"], b["q"]) and np.array_equal(a["t"], b["t"]) and a["J"] == b["J"]
                   for a, b in zip(plain, burst)) and \
            all(np.array_equal(a["q"], b["q"]) and a["J"] == b["J"] for a, b in zip(plain, poisson))
        lat = np.array([r["latency_ms"] for r in poisson])
        evals = sum(ng + nl for _, ng, nl in reqs)
        return {"requests": len(req_t), "evals": evals,
                "mix": "N uniform over {32,64,96,128}, 100-2000 poses, r 0.5-1.5 mm, 1000-4000 + 25% rotations, top-8",
                "plain_regs_per_s": round(len(req_t) / t_plain, 3),
                "served_regs_per_s": round(len(req_t) / t_burst, 3),
                "served_vs_plain": round(t_plain / t_burst, 3),
                "poisson_rate_per_s": round(rate, 3), "poisson_regs_per_s": round(len(req_t) / t_pois, 3),
                "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
                "p999_ms": round(float(np.percentile(lat, 99.9)), 2), "results_equal_plain": bool(same)}
    finally:
        for ob, sw in handles:
            ob.close()
            sw.close()


# Per-rotation counters of the search kernels as they are now, from one ncu capture each of an
# 8-rotation launch of `bench.py --ncu-case` (dram__bytes_read.sum + dram__bytes_write.sum, and
# smsp__inst_executed.sum for the voxeliser); a launch of B rotations is scaled from them by B/8
# (the z pass adds one spectrum read per launch).  A kernel changed since its capture has no entry.
NCU_DRAM_BYTES_PER_ROT = {"plane": (545298176 + 3637760) / 8, "fwd2d": (18521856 + 229523456) / 8,
                          "zpass": (340853760 - 68157440 + 489946880) / 8, "voxelise": (1056256 + 0) / 8}
NCU_WARP_INST_PER_ROT = {"voxelise": 343219446 / 8}
# SMs x warp schedulers: one warp instruction issued per scheduler per clock
ISSUE_SLOTS = 152 * 4


def max_over_ranks(ms, ws, device):
    """The slowest rank's timed milliseconds (every rank gets the same value)."""
    if ws <= 1:
        return ms
    import torch
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(ws, units_per_rank, ms_max):
    """Units all ranks processed / the slowest rank's time (weak scaling: each
    rank runs its own replica of the workload)."""
    return ws * units_per_rank / (ms_max / 1000.0)


class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def model_bytes_per_eval(N):
    """Bytes one rotation moves through HBM in the 5-pass pruned FFT model
    (x-pass write, y-pass read+write, z-pass read, spectrum read, z-pass
    write, inverse-y read+write, inverse-x read)."""
    M = 2 * N
    H = M * M * (M // 2 + 1) * 8
    return (N * N * (M // 2 + 1) * 8) * 2 + (M * N * (M // 2 + 1) * 8) * 2 + H + H + 2 * H + H


def kernel_bytes(name, N):
    """Compulsory HBM bytes per rotation of each fused search kernel (inputs
    read once, outputs written once), P = M/2 + 2 complex per row."""
    M = 2 * N
    P = M // 2 + 2
    y = N * M * P * 8
    z = M * M * P * 8
    bits = N * N * N // 8
    return {"voxelise": bits, "fwd2d": bits + y, "zpass": y + z, "plane": z}.get(name)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sm_max_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("sm_max_mhz", 2070.0))
    return 2070.0


_ORACLE_GRID = {}


def cpu_oracle_rate(w, n_rot, seed=0, workers=1):
    """The FP64 oracle's search (sweep + FFT correlation + argmax per rotation)
    on a bounded sample of rotations of the same workload, its rotations spread
    over `workers` host threads; returns (evals/s, seconds, rotations)."""
    import oracle as O
    if id(w) not in _ORACLE_GRID:   # the object set-up is not part of an eval
        _ORACLE_GRID[id(w)] = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)[:2]
    Go, oo = _ORACLE_GRID[id(w)]
    from paper_2605_21398_gb300 import synth
    quats = synth.random_unit_quats(n_rot, 1234 + seed)
    t0 = time.perf_counter()
    O.search_peaks(Go, w.poses_world, quats, w.h, w.N, w.radius, w.length, workers=workers)
    dt = time.perf_counter() - t0
    return n_rot / dt, dt, n_rot


def run_reference(args):
    rank, ws = _dist()
    if rank != 0:
        return 0
    from paper_2605_21398_gb300 import synth
    w = synth.make_workload(WORKLOAD)
    cores = os.cpu_count() or 1
    per_step = 2 * cores
    for _ in range(args.warmup):
        cpu_oracle_rate(w, cores, workers=cores)
    times = []
    for s in range(args.steps):
        r, dt, n = cpu_oracle_rate(w, per_step, seed=s, workers=cores)
        times.append(dt)
    total = per_step * args.steps
    value = total / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "large128: 128^3 lattice at 0.15 mm (canvas 256^3), 5000 probe poses on 3 raster "
                                   "segments (20% labels flipped, 0.02 mm noise), 65k-triangle star object; the oracle's "
                                   "per-rotation search (sweep + FP64 FFT correlation + argmax) on sampled rotations",
                       "sample": "%d rotations per step" % per_step},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": "%d random rotations per step over %d host threads, sweep + FFT correlation "
                                       "+ argmax" % (per_step, cores)},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ncu_case(variant="plain"):
    """One search of 8 SF rotations in one batch on the bench workload (every
    search kernel launches once with 8 rotations, a few GB on the device), then
    a refinement of 8 candidates near the planted pose.  variant: "plain", or
    the search with the rotated object ("rotate_object") or the label-aware
    score ("label_aware"), or the z pass with its DFT stages on the tensor
    cores ("zpass_tc")."""
    from paper_2605_21398_gb300 import build, dock, synth
    build.build()
    w = synth.make_workload(WORKLOAD)
    ctx = dock.Context(0)
    ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
    if variant == "rotate_object":
        sw.set_rotate_object(True)
    elif variant == "label_aware":
        sw.set_label_aware(True)
    elif variant == "zpass_tc":
        ctx.set_tuning(N=w.N, zpass_cols=16, zpass_tc=1)
    elif variant != "plain":
        raise ValueError("unknown ncu variant %r" % variant)
    c = ctx.search_so3(ob, sw, 8, 4, batch=8)
    # refinement of 8 candidates near the planted pose (every refinement kernel launches)
    rng = np.random.default_rng(3)
    cands = []
    for _ in range(8):
        dq = synth.axis_angle_quat(np.radians(rng.normal(0.0, 1.0, 3)))
        cands.append(dict(q=synth.quat_mul(dq, w.gt_q), t=w.gt_t + rng.normal(0.0, 0.05, 3)))
    r = ctx.refine_se3(ob, sw, cands)
    print(json.dumps({"ncu_case": WORKLOAD, "variant": variant, "rotations": 8, "best_score": c[0]["score"],
                      "refined": len(r)}))
    ob.close()
    sw.close()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--n-global", type=int, default=N_GLOBAL)
    ap.add_argument("--n-local", type=int, default=N_LOCAL)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--ncu-variant", default="plain", choices=["plain", "rotate_object", "label_aware", "zpass_tc"])
    ap.add_argument("--batch-study", type=int, default=0, metavar="N_REQ",
                    help="time dock_register_batch against the plain loop on N_REQ requests of the batched mix")
    ap.add_argument("--serving-study", type=int, default=0, metavar="N_REQ",
                    help="Poisson arrivals of N_REQ requests at 1, 2 and 4 req/s: regs/s and latency percentiles")
    ap.add_argument("--ncu-case", action="store_true",
                    help="small fixed case for ncu captures: one search of 8 rotations (batch 8) of the bench workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return run_ncu_case(args.ncu_variant)
    if args.batch_study or args.serving_study:
        from paper_2605_21398_gb300 import build, dock, synth
        build.build()
        ctx = dock.Context(0)
        out = {}
        if args.batch_study:
            out["batch_study"] = batch_study(ctx, synth, args.batch_study)
        if args.serving_study:
            out["serving_study"] = serving_study(ctx, synth, args.serving_study, (1.0, 2.0, 4.0))
        ctx.close()
        print(json.dumps(out))
        return 0

    import torch
    rank, ws = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2605_21398_gb300 import build, dock, synth
    build.build()

    w = synth.make_workload(WORKLOAD, replicate=rank)
    stream = torch.cuda.Stream()
    ctx = dock.Context(local, 0, stream.cuda_stream)
    t0 = time.perf_counter()
    ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    obj_setup_ms = 1000 * (time.perf_counter() - t0)
    sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
    # launch shape of the search kernels for this lattice side, picked by the
    # autotuner (once per lattice side, before the warm-up; results do not
    # depend on it)
    tuning = ctx.autotune(ob, sw, n_rot=512)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def step():
        return ctx.register(ob, sw, args.n_global, args.n_local, THETA, TOP_K)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.reset_kernel_stats()
    ctx.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    ms_steps = []
    results = []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        results.append(step())
        ev1.record(stream)
        ev1.synchronize()
        ms_steps.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ctx.set_profiling(False)
    stats = ctx.kernel_stats()
    ms_total = max_over_ranks(float(sum(ms_steps)), ws, "cuda")
    evals_per_step = args.n_global + args.n_local
    value = whole_job_rate(ws, evals_per_step * args.steps, ms_total)

    # roofline of the dominant HBM-bound search kernel (algorithmic bytes per
    # launch / its average CUDA-event duration); every kernel's share is listed
    peak, peak_src = load_peaks()
    rot_total = evals_per_step * args.steps
    kernels = {k: {"launches": v[0], "total_ms": round(v[1], 3)} for k, v in stats.items()}
    tot_all = sum(v[1] for v in stats.values()) or 1.0
    for k in kernels:
        kernels[k]["share"] = round(stats[k][1] / tot_all, 4)
    def hbm_roofline(k):
        launches, tot_ms = stats[k]
        M = 2 * w.N
        P = M // 2 + 2
        total_bytes = kernel_bytes(k, w.N) * rot_total
        if k == "zpass":
            total_bytes += M * M * P * 8 * launches   # spectrum read once per launch (block column)
        achieved = total_bytes / (tot_ms / 1000.0) / 1e9
        rot_per_launch = rot_total / max(1, launches)
        traffic = None
        if k in NCU_DRAM_BYTES_PER_ROT:
            traffic = NCU_DRAM_BYTES_PER_ROT[k] * rot_per_launch + (M * M * P * 8 if k == "zpass" else 0)
        return {"bound": "hbm", "kernel": k, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": int(traffic) if traffic else None,
                "traffic_source": "ncu capture of an 8-rotation launch, scaled to %.1f rotations per launch"
                                  % rot_per_launch, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": int(total_bytes / max(1, launches))}

    def issue_roofline(k):
        # the voxeliser moves almost no data: it is bound by instruction issue
        launches, tot_ms = stats[k]
        inst = NCU_WARP_INST_PER_ROT[k] * rot_total
        achieved = inst / (tot_ms / 1000.0) / 1e9
        pk = ISSUE_SLOTS * sm_max_mhz() / 1e3
        return {"bound": "alu", "kernel": k, "achieved": round(achieved, 1), "peak": round(pk, 1),
                "unit": "G warp-instructions/s", "frac": round(achieved / pk, 4),
                "traffic": int(NCU_DRAM_BYTES_PER_ROT[k] * rot_total / max(1, launches)),
                "work_source": "smsp__inst_executed.sum of an 8-rotation ncu capture (%.1f M per rotation)"
                               % (NCU_WARP_INST_PER_ROT[k] / 1e6),
                "peak_source": "152 SMs x 4 schedulers x %.0f MHz (maximum SM clock)" % sm_max_mhz()}

    search = {k: stats[k][1] for k in ("voxelise", "fwd2d", "zpass", "plane") if k in stats}
    hbm = {k: v for k, v in search.items() if k != "voxelise"}
    dom = max(search, key=lambda k: search[k]) if search else None
    dom_hbm = max(hbm, key=lambda k: hbm[k]) if hbm else None
    roofline = roofline_hbm = None
    if dom:
        roofline = issue_roofline(dom) if dom == "voxelise" else hbm_roofline(dom)
        roofline["dominant_overall"] = max(stats, key=lambda k: stats[k][1])
    if dom_hbm:
        roofline_hbm = hbm_roofline(dom_hbm)
    model_frac = value / ws * model_bytes_per_eval(w.N) / (peak * 1e9)

    # end-to-end through the public API from host buffers (object + sweep + register + result)
    e2e = None
    if not args.no_e2e:
        h2d = w.obj.verts.nbytes + w.obj.tris.astype(np.int32).nbytes + w.poses_world.nbytes + w.labels.nbytes
        d2h = 176
        t_e = []
        for s in range(max(1, min(2, args.steps))):
            torch.cuda.synchronize()
            ta = time.perf_counter()
            ob2 = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
            sw2 = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
            ctx.register(ob2, sw2, args.n_global, args.n_local, THETA, TOP_K)
            t_e.append(time.perf_counter() - ta)
            ob2.close()
            sw2.close()
        e2e = {"value": evals_per_step * len(t_e) / sum(t_e), "unit": "evals/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": d2h}

    # variants of the search on the same registration (one warm-up, one
    # timed step each): the label-aware score (the 20 % non-contact-labelled
    # poses score min(O, 0)) and the rotated-object mechanism of Sec. IV-D
    def variant(switch, kernel_names, params=None):
        sw_v = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
        switch(sw_v)
        ctx.register(ob, sw_v, args.n_global, args.n_local, THETA, TOP_K, params=params)
        torch.cuda.synchronize()
        ctx.reset_kernel_stats()
        ctx.set_profiling(True)
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        r_v = ctx.register(ob, sw_v, args.n_global, args.n_local, THETA, TOP_K, params=params)
        ev1.record(stream)
        ev1.synchronize()
        ms_v = ev0.elapsed_time(ev1)
        ctx.set_profiling(False)
        st_v = ctx.kernel_stats()
        sw_v.close()
        out = {"value": evals_per_step / (ms_v / 1000.0), "unit": "evals/s", "ms_per_step": round(ms_v, 2),
               "ms_per_eval_search": round(sum(st_v[k][1] for k in kernel_names if k in st_v) / evals_per_step
                                           * 1000.0, 3),
               "kernels_ms": {k: round(st_v[k][1], 2) for k in kernel_names if k in st_v},
               "best_search_rot": int(r_v["best_search"]["rot"]), "J": r_v["J"]}
        return out, r_v

    label_aware = rotate_object = lbfgsb = None
    r_la = r_ro = r_lb = None
    if rank == 0 and not args.no_variants:
        label_aware, r_la = variant(lambda sv: sv.set_label_aware(True),
                                    ("voxelise", "voxelise_nc", "fwd2d", "fwd2d_nc", "zpass_dual", "plane"))
        label_aware["non_contact_poses"] = int((w.labels == 0).sum())
        rotate_object, r_ro = variant(lambda sv: sv.set_rotate_object(True),
                                      ("voxelise", "resample", "fwd2d", "zpass", "plane"))
        # the refinement by L-BFGS-B (Sec. V-C as printed) instead of Gauss-Newton
        p_lb = dock.default_params()
        p_lb.solver = dock.SOLVER_LBFGSB
        p_lb.iters = 200
        lbfgsb, r_lb = variant(lambda sv: None, ("refine_eval", "refine_lbfgs", "refine_solve"), params=p_lb)
        lbfgsb["refine_ms"] = round(sum(lbfgsb["kernels_ms"].values()), 2)
        del lbfgsb["ms_per_eval_search"]

    cufft = None
    if rank == 0 and not args.no_variants:
        try:
            cufft = cufft_comparison(ctx, ob, sw, w, stream)
            ours = sum(stats[k][1] for k in ("fwd2d", "zpass", "plane") if k in stats) / rot_total * 1000.0
            cufft["ours_fwd2d_zpass_plane_us_per_rotation"] = round(ours, 1)
        except Exception as exc:   # reported, not fatal to the throughput line
            cufft = {"error": "%s: %s" % (type(exc).__name__, exc)}

    serving = None
    if rank == 0 and not args.no_serving:
        try:
            serving = serving_experiment(ctx, synth)
        except Exception as exc:   # reported, not fatal to the throughput line
            serving = {"error": "%s: %s" % (type(exc).__name__, exc)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's search on every host core (rotations spread over threads),
        # and on one core
        cores = os.cpu_count() or 1
        r, dt, n = cpu_oracle_rate(w, 2 * cores, workers=cores)
        r1, dt1, n1 = cpu_oracle_rate(w, 3, seed=1)
        cpu = {"value": r, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "%d random rotations of the same workload over %d host threads (sweep + FP64 FFT "
                         "correlation + argmax), %.1f s" % (n, cores, dt),
               "single_core": {"value": r1, "unit": "evals/s", "cores": 1,
                               "sample": "%d random rotations, %.1f s" % (n1, dt1)}}

    a = np.asarray(w.obj.verts).min(0) * 0.5 + np.asarray(w.obj.verts).max(0) * 0.5
    res = results[-1]
    Rr, Rg = synth.quat_to_mat(res["q"]), synth.quat_to_mat(w.gt_q)
    err_t = float(np.linalg.norm(Rr @ a + res["t"] - (Rg @ a + w.gt_t)))
    err_r = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(Rr @ Rg.T) - 1) / 2))))
    for vd, rv in ((label_aware, r_la), (rotate_object, r_ro), (lbfgsb, r_lb)):
        if vd is not None:
            Rl = synth.quat_to_mat(rv["q"])
            vd["trans_err_mm"] = round(float(np.linalg.norm(Rl @ a + rv["t"] - (Rg @ a + w.gt_t))), 4)
            vd["rot_err_deg"] = round(math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(Rl @ Rg.T) - 1) / 2)))), 4)
    launches = int(sum(v[0] for v in stats.values()))
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "large128: 128^3 lattice at 0.15 mm (canvas 256^3), %d SF + %d GeoBall-SF "
                                   "rotations, 5000 probe poses on 3 raster segments (20%% labels flipped, 0.02 mm "
                                   "noise), 65k-triangle star object, top-%d refined (20 Gauss-Newton iterations)"
                                   % (args.n_global, args.n_local, TOP_K),
                       "l2": "inputs larger than L2 (per-batch FFT intermediates ~13 GB) and a 256 MB L2 flush "
                             "before every step",
                       "parallelism": "replicas" if ws > 1 else "single",
                       "search_launch_shape": {k: tuning[k] for k in ("batch", "group", "vox_blocks", "plane_cl",
                                                                      "plane_tma", "fwd_runs", "zpass_cols", "zpass_tc",
                                                                      "fft_plan")}},
            "roofline": roofline, "roofline_hbm": roofline_hbm, "model_roofline_frac": round(model_frac, 4),
            "model_bytes_per_eval": model_bytes_per_eval(w.N),
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "kernels": kernels,
            "ms_per_eval_search": round(sum(stats[k][1] for k in ("voxelise", "fwd2d", "zpass", "plane") if k in stats)
                                        / rot_total * 1000.0, 3),
            "clocks": clk, "object_setup_ms": round(obj_setup_ms, 2), "serving": serving,
            "label_aware": label_aware, "rotate_object": rotate_object, "lbfgsb_refinement": lbfgsb,
            "cufft_comparison": cufft,
            "accuracy": {"trans_err_mm": round(err_t, 4), "rot_err_deg": round(err_r, 4), "J": res["J"]}}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
