"""Throughput benchmark of the KiloNeuS sphere-traced render path (one JSON line on rank 0).

Default step: one BF16 render of the 1080p precision-form workload -- the 32^3 Kilo-grid (32768 cells,
3 hidden layers of width 64, 128^3 occupancy mask) from 8 seeded orbit cameras at 1920x1080, max 128
steps, eps 1e-4: 16.6 M primary rays, sphere-traced on the tensor cores (split-BF16 products, FP32
accumulation), the last step, the normal and the colour in FP32 (kns_render, precision KNS_BF16).  The
grid is resident in HBM before timing starts.  Each timed step is bracketed by CUDA events on the
launching stream; between steps a 512 MiB buffer is overwritten to flush the 126 MB L2, outside the
events.  The same line carries the plain FP32 GPU path on the same workload (same protocol), the
speed-up, the BF16 error against the FP64 oracle on sampled pixels (hit agreement; depth, RGB and
normal-angle quantiles and the fractions within the stated gates), the serving stream's p50/p99
latency at four Poisson rates, the roofline of the dominant kernel against peaks measured on the GPU,
the end-to-end rate through host buffers, and the oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
                    [--workload c3l|c3s|c2|c1|train|pt] [--impl kns|reference] [--serving 0|1]

--workload train times the NeuS-style training step instead (kns_train_step: loss and hand-written
backward): 2^18 rays x (64 stratified + 32 importance samples) through the 16^3 grid (3 hidden
layers of width 32), L1 colour + 0.1 x eikonal on 2^16 points; targets are renders of a perturbed
sphere grid by the render path; metric Mrays/s through the step.  --workload pt times Lambertian path
tracing (kns_path_trace) of the 16^3 grid: 800x800, 16 paths per pixel, up to 4 traces per path.

Multi-GPU (torchrun): every rank renders its own batch on its own GPU (replicas, no
collective on the data path); value = rays of all ranks / max-over-ranks time.
`--impl reference` times the FP64 CPU oracle on this host's cores on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s sphere-traced+shaded, BF16 vs FP32 at stated error; serving p50/p99 ms"
UNIT = "Mrays/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kns", choices=["kns", "reference"])
    ap.add_argument("--workload", default="c3l")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true", help="BF16: skip the FP32 render of the same workload")
    ap.add_argument("--no-accuracy", action="store_true", help="BF16: skip the sampled comparison with the oracle")
    ap.add_argument("--serving", type=int, default=1, help="BF16: also run the serving stream (0 = skip)")
    ap.add_argument("--serving-rates", type=float, nargs="+", default=[50, 100, 200, 400])
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cams", type=int, default=0, help="use only the first N cameras (small profiling cases)")
    ap.add_argument("--train-rays", type=int, default=0,
                    help="train workload: rays per step (eikonal points scale along; small profiling cases)")
    ap.add_argument("--tune", default="off", choices=["cache", "force", "off"],
                    help="schedule autotuning of the timed precision before timing (the cached best, tuning once "
                         "if absent; re-tune; or the library defaults, picked by sweeps at these workloads)")
    return ap.parse_args()


def workload_config(name, desc, cams, W, H, ms, eps, precision):
    return {"workload": "%s: %d^3 Kilo-grid, SDF MLP %d hidden x %d (softplus beta=%g, PE L=%d), colour MLP "
                        "%d hidden x %d, occupancy %s; %d orbit cameras x %dx%d, max %d steps, eps %g; %s"
                        % (name, desc.N, desc.sdf_hidden, desc.sdf_width, desc.softplus_beta, desc.pe_pos_L,
                           desc.col_hidden, desc.col_width,
                           ("%d^3" % desc.occ_res) if desc.occ_res else "none",
                           cams.shape[0], W, H, ms, eps, precision),
            "rays_per_step": int(cams.shape[0] * W * H), "grid": "%d^3" % desc.N, "sdf_width": desc.sdf_width,
            "sdf_hidden": desc.sdf_hidden, "resolution": "%dx%d" % (W, H), "n_cameras": int(cams.shape[0]),
            "max_steps": ms, "eps": eps, "precision": precision,
            "l2": "flushed between steps (512 MiB write outside the timed events)",
            "inputs": "synthetic grid: SAL geometric initialisation for a sphere of radius 0.5 (seed 0) plus per-cell "
                      "N(0, 1e-3) perturbation, seeded orbit cameras"}


def mac_counts(desc):
    """Algorithmic multiply-adds: per trace sample (d only) and per hit (full SDF + gradient + colour)."""
    IN = 3 + 6 * desc.pe_pos_L
    Wd, Hd = desc.sdf_width, desc.sdf_hidden
    trace = IN * Wd + (Hd - 1) * Wd * Wd + Wd
    full_fwd = IN * Wd + (Hd - 1) * Wd * Wd + Wd * (1 + desc.feat_dim)
    bwd = (Hd - 1) * Wd * Wd + IN * Wd
    cin = desc.feat_dim + 3 + 3 + 6 * desc.pe_dir_L + (3 if desc.col_use_x else 0)
    colour = cin * desc.col_width + desc.col_width * 3
    return trace, full_fwd + bwd + colour


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# the sources each profiled kernel is compiled from: a committed capture counts only while they are unchanged
KERNEL_SOURCES = {
    "trace_tc_kernel": ["kns_tc.cu", "kns_tc.cuh", "kns_wave.cuh", "kns_device.cuh", "kns_kernels.h"],
    "wave_eval_block_kernel": ["kns_wave.cu", "kns_wave.cuh", "kns_device.cuh", "kns_kernels.h"],
    "k_tile_backward": ["kns_train_tile.cu", "kns_train.cuh", "kns_device.cuh", "kns_kernels.h"],
}


def profile_traffic(kernel_tag: str):
    """DRAM bytes per full launch from the committed ncu summary tagged kernel_tag, if the sources of
    its kernel still hash to the summary's kernel_source_sha1 (else None: the counters are stale)."""
    src_hash = kernel_source_hash(kernel_tag)
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        text = open(os.path.join(pdir, fn)).read()
        m_tag = re.search(r"kernel_tag:\s*(\S+)", text)
        m_hash = re.search(r"kernel_source_sha1:\s*([0-9a-f]+)", text)
        m_b = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
        if m_tag and m_hash and m_b and m_tag.group(1) == kernel_tag and m_hash.group(1) == src_hash:
            return float(m_b.group(1))
    return None


def kernel_source_hash(kernel_tag: str) -> str:
    """sha1 over the kernel's source files (KERNEL_SOURCES, in that order), or over every csrc file."""
    cdir = os.path.join(ROOT, "paper_2206_10885_gb300", "csrc")
    files = next((v for k, v in KERNEL_SOURCES.items() if kernel_tag.startswith(k)), None)
    if files is None:
        files = sorted(fn for fn in os.listdir(cdir) if fn.endswith((".cu", ".cuh", ".h")))
    h = hashlib.sha1()
    for fn in files:
        h.update(open(os.path.join(cdir, fn), "rb").read())
    return h.hexdigest()


def max_over_ranks(vals, device, world: int):
    """Element-wise maximum of per-rank values (the slowest rank's times); identity for one rank."""
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(units_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Units of all ranks per second (millions) over the slowest rank's time: weak-scaling value."""
    return world * units_per_rank * steps / (total_ms * 1e-3) / 1e6


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(desc, w, cams, W, H, ms, eps, seconds: float, seed: int = 0):
    """Times the FP64 oracle (as it stands) on a seeded random sample of the workload's rays."""
    import oracle as O
    occ = O.occupancy(desc, w) if desc.occ_res else None
    n_pix = cams.shape[0] * W * H
    rng = np.random.default_rng(seed)
    done, elapsed, batch = 0, 0.0, 4096
    while elapsed < seconds:
        sel = np.sort(rng.integers(0, n_pix, batch))
        t0 = time.perf_counter()
        O.render(desc, w, occ, cams, W, H, ms, eps, sel=sel)
        dt = time.perf_counter() - t0
        elapsed += dt
        done += batch
        if dt < seconds / 8:
            batch *= 2
    return done / elapsed / 1e6, done, elapsed, O.num_threads()


def run_reference(args, rank, world):
    from paper_2206_10885_gb300 import synth as S
    if rank != 0:
        return
    desc, w, cams, W, H, ms, eps = S.workload(args.workload)
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_rate(desc, w, cams, W, H, ms, eps, 0.2)
    vals = []
    total_rays, total_s, cores = 0, 0.0, 1
    for k in range(args.steps):
        v, n, s, cores = oracle_rate(desc, w, cams, W, H, ms, eps, per_step, seed=k + 1)
        vals.append(v)
        total_rays += n
        total_s += s
    value = total_rays / total_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cams.shape[0] * W * H / (value * 1e6), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, desc, cams, W, H, ms, eps, "fp64 oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d rays drawn (seeded, with replacement) from the workload's rays over "
                                       "%d steps (%.1f s)"
                                       % (total_rays, args.steps, total_s)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def bf16_accuracy(O, desc, w, occ, cams, W, H, ms, eps, bf, fp, n_random=4000, n_hits=4000, seed=4):
    """BF16 render vs the FP64 oracle on sampled pixels (seeded: random pixels plus pixels the BF16 or
    FP32 render hit): hit agreement, and on pixels both hit the error quantiles and the fraction within
    each gate (depth 1e-3, RGB 1/255, normal angle 0.5 degrees)."""
    rng = np.random.default_rng(seed)
    n_pix = bf["hit"].shape[0]
    hits = np.where((bf["hit"] == 1) | (fp["hit"] == 1))[0]
    sel = np.unique(np.concatenate([rng.integers(0, n_pix, n_random),
                                    hits[rng.integers(0, max(1, hits.size), n_hits)] if hits.size else []]).astype(np.int64))
    o = O.render(desc, w, occ, cams, W, H, ms, eps, sel=sel)
    g = {k: v[sel] for k, v in bf.items()}
    gh, oh = g["hit"] == 1, o["hit"] == 1
    both = gh & oh
    dd = np.abs(g["depth"][both].astype(np.float64) - o["depth"][both])
    dr = np.abs(g["rgb"][both].astype(np.float64) - o["rgb"][both]).max(axis=1)
    ang = np.degrees(np.arccos(np.clip(np.sum(g["normal"][both].astype(np.float64) * o["normal"][both], axis=1), -1, 1)))
    q = lambda a: {"p50": float(np.quantile(a, 0.5)), "p99": float(np.quantile(a, 0.99)),
                   "p99.9": float(np.quantile(a, 0.999)), "max": float(a.max())} if a.size else None
    return {"pixels": int(sel.size), "both_hit": int(both.sum()), "hit_agreement": float(np.mean(gh == oh)),
            "depth_within_1e-3": float(np.mean(dd <= 1e-3)) if dd.size else None,
            "rgb_within_1/255": float(np.mean(dr <= 1 / 255)) if dr.size else None,
            "normal_within_0.5deg": float(np.mean(ang <= 0.5)) if ang.size else None,
            "depth_err": q(dd), "rgb_err": q(dr), "normal_angle_deg": q(ang),
            "sample": "%d random pixels + %d drawn from pixels either render hit (seed %d), all %d cameras"
                      % (n_random, n_hits, seed, cams.shape[0])}


def serving_run(kns, S, main_grid, rates, seconds, slots=3):
    """The serving workload: 4 resident BF16 grids (2 x 16^3 width 32, 2 x 32^3 width 64), Poisson
    arrivals at each rate, resolutions uniform over {256^2, 512^2, 800^2, 1920x1080}; p50/p99 latency
    and delivered Mrays/s per rate."""
    from paper_2206_10885_gb300 import serve
    grids = {"c3s-0": (S.config_desc("c3s"), S.sal_sphere_grid(S.config_desc("c3s"), seed=0)),
             "c3s-1": (S.config_desc("c3s"), S.sal_sphere_grid(S.config_desc("c3s"), seed=1)),
             "c3l-0": main_grid,
             "c3l-1": (S.config_desc("c3l"), S.sal_sphere_grid(S.config_desc("c3l"), seed=1))}
    server = serve.RenderServer(grids, slots=slots, precision=kns.KNS_BF16)
    names = list(grids)
    out = []
    try:
        warm = [serve.Request(-1 - k, names[k % len(names)], S.orbit_cameras(1, 1920, 1080, seed=k)[0], 1920, 1080)
                for k in range(len(names) * slots)]
        for r in warm:
            server.submit(r)
        server.drain()
        for rate in rates:
            n = max(8, int(rate * seconds))
            stream = serve.poisson_stream(n, rate, seed=int(rate), grids=names, resolutions=serve.RES_MIX)
            res = serve.run_stream(server, stream)
            out.append({"rate_per_s": rate, "requests": res["requests"], "p50_ms": res["p50_ms"],
                        "p99_ms": res["p99_ms"], "mrays_per_s": res["mrays_per_s"], "batches": res["batches"],
                        "batches_with_two_grids": res["mixed_batches"]})
    finally:
        server.close()
    return {"grids": "2 x 16^3/w32 + 2 x 32^3/w64, BF16, resident, stacked per shape (a batch may hold both grids "
                     "of a shape)", "resolutions": "256^2, 512^2, 800^2, 1920x1080",
            "arrivals": "Poisson, %.1f s per rate" % seconds, "slots": slots, "per_rate": out}


def run_kns(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_2206_10885_gb300 as kns
    from paper_2206_10885_gb300 import build as kbuild
    from paper_2206_10885_gb300 import synth as S

    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2206_10885_gb300", "libkns.so")):
        kbuild.build()
    if world > 1:
        dist.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    desc, w, cams, W, H, ms, eps = S.workload(args.workload)
    if args.cams:
        cams = cams[:args.cams]
    precision = kns.KNS_BF16 if args.precision == "bf16" else kns.KNS_FP32
    ctx = kns.Context(local_rank)
    grid = kns.Grid.load(ctx, desc, w)  # occupancy mask built on the device, untimed
    n_rays = cams.shape[0] * W * H
    stream = torch.cuda.current_stream()
    frame = kns.alloc_frame(n_rays, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    props = torch.cuda.get_device_properties(local_rank)

    tuning = None
    if args.tune != "off":
        from paper_2206_10885_gb300 import autotune
        tuning, tuned_ms, tried = autotune.tune(ctx, grid, cams, W, H, ms, eps, precision,
                                                use_cache=args.tune == "cache")
        if rank == 0 and tried:
            print("# autotune: %d settings, best %s at %.3f ms" % (len(tried), tuning, tuned_ms), file=sys.stderr)

    def render(prec, tun=None):
        kns.render(ctx, grid, cams, W, H, ms, eps, precision=prec, out=frame, stream=stream, tuning=tun)

    def timed(prec, tun, steps):
        """steps renders, each bracketed by CUDA events on the launching stream, L2 flushed between."""
        for _ in range(max(3, args.warmup)):
            render(prec, tun)
        ctx.sync(stream)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            render(prec, tun)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ctx.sync(stream)
        return [a.elapsed_time(b) for a, b in evs]

    def stats_of(prec, tun):
        render(prec, dict(tun or {}, timing=1))
        ctx.sync(stream)
        return ctx.render_stats(), ctx.round_trace()

    clocks = ClockSampler(local_rank).start() if rank == 0 else None
    times = timed(precision, tuning, args.steps)
    clock_info = clocks.stop() if clocks else None
    total_ms = sum(times)
    main_out = {k: v.cpu().numpy() for k, v in frame[0].items()}
    st, trace = stats_of(precision, tuning)

    # the plain FP32 GPU path on the same workload, same protocol (the comparison the metric names)
    fp32 = None
    if precision == kns.KNS_BF16 and not args.no_fp32_compare:
        t32 = timed(kns.KNS_FP32, None, max(3, args.steps // 2))
        fp32_out = {k: v.cpu().numpy() for k, v in frame[0].items()}
        st32, _ = stats_of(kns.KNS_FP32, None)
        (t32_ms,) = max_over_ranks([sum(t32)], dev, world)
        fp32 = {"value": whole_job_rate(n_rays, world, len(t32), t32_ms), "unit": UNIT,
                "ms_per_step": t32_ms / len(t32), "steps": len(t32),
                "phases_ms_per_render": {k: st32[k] for k in ("ms_generate", "ms_sort", "ms_eval_fp32", "ms_shade",
                                                              "ms_total")},
                "counts_per_render": {k: st32[k] for k in ("rounds", "hits", "samples_fp32", "samples_tail")}}

    # e2e through the public API: cameras from host memory, outputs read back to pinned host buffers
    host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in frame[0].items()
            if k in ("rgb", "depth", "normal", "hit")}
    d2h = sum(v.numel() * v.element_size() for v in host.values())
    h2d = cams.nbytes
    for _ in range(2):
        render(precision, tuning)
        for k, v in host.items():
            v.copy_(frame[0][k], non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        render(precision, tuning)
        for k, v in host.items():
            v.copy_(frame[0][k], non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0

    total_ms, e2e_s = max_over_ranks([total_ms, e2e_s], dev, world)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(n_rays, world, args.steps, total_ms)
    e2e_value = whole_job_rate(n_rays, world, args.steps, e2e_s * 1e3)

    if rank == 0:
        import oracle as O
        mp = load_peaks()
        pk = ctx.measure_peaks(stream)
        p_ffma, p_mufu = pk["ffma_flops"] / 1e12, pk["mufu_ops"] / 1e9  # TFLOP/s, Gop/s
        mac_trace, mac_hit = mac_counts(desc)
        IN = 3 + 6 * desc.pe_pos_L
        Wd, Hd = desc.sdf_width, desc.sdf_hidden
        mac_tc = IN * Wd + (Hd - 1) * Wd * Wd  # hidden layers of a trace sample (the d row is FP32)
        transc = 2 * Hd * Wd  # ex2 + lg2 per hidden unit (softplus)
        hbm = float(mp.get("hbm_gbs", 6772.9))
        bf16_peak = float(mp.get("bf16_tflops", 1944.1))
        if precision == kns.KNS_BF16:
            # dominant kernel: the persistent tensor-core trace (every BF16 round, sort and scatter inside)
            S_ = st["samples_bf16"]
            kms = st["ms_eval_bf16"]
            t_mufu = S_ * transc / (p_mufu * 1e9) * 1e3
            t_tc = 2.0 * S_ * mac_tc / (bf16_peak * 1e12) * 1e3
            achieved = S_ * transc / (kms * 1e-3) / 1e9 if kms > 0 else 0.0
            roof = {"bound": "alu", "kernel": "trace_tc_kernel (persistent BF16 trace)", "unit": "Gop/s",
                    "peak": p_mufu, "achieved": achieved, "frac": achieved / p_mufu,
                    "peak_source": "measured on this GPU: ex2.approx micro-kernel (kns_measure_peaks), of measured",
                    "work": "2 MUFU (ex2, lg2) per hidden unit x %d units per sample x %d BF16 samples" % (Hd * Wd, S_),
                    "kernel_ms_per_render": kms,
                    "tensor_pipe_frac": 2.0 * S_ * mac_tc / (kms * 1e-3) / (bf16_peak * 1e12) if kms > 0 else 0.0,
                    "tensor_pipe_note": "algorithmic hidden-layer FLOP (2 x %d MAC per sample) over the kernel time, "
                                        "of measured bf16 %.1f TFLOP/s; the split issues 3x that on padded K" % (mac_tc, bf16_peak),
                    "t_floor_ms": max(t_mufu, t_tc), "t_floor_terms_ms": {"mufu": t_mufu, "tensor": t_tc},
                    "traffic": profile_traffic("trace_tc_kernel_bf16_%s" % args.workload)}
        else:
            S_ = st["samples_fp32"]
            kms = st["ms_eval_fp32"]
            flops = 2.0 * S_ * mac_trace
            achieved = flops / (kms * 1e-3) / 1e12 if kms > 0 else 0.0
            t_ffma = flops / (p_ffma * 1e12) * 1e3
            t_mufu = S_ * transc / (p_mufu * 1e9) * 1e3
            roof = {"bound": "alu", "kernel": "wave_eval_block_kernel + wave_tail_warp_kernel (FP32 evaluation class)",
                    "unit": "TFLOP/s", "peak": p_ffma, "achieved": achieved, "frac": achieved / p_ffma,
                    "peak_source": "measured on this GPU: FFMA micro-kernel (kns_measure_peaks), of measured",
                    "kernel_ms_per_render": kms, "flop_per_sample": 2 * mac_trace,
                    "t_floor_ms": max(t_ffma, t_mufu), "t_floor_terms_ms": {"ffma": t_ffma, "mufu": t_mufu},
                    "traffic": profile_traffic("wave_eval_block_kernel_fp32_%s" % args.workload)}
        roof["measured_peaks"] = {"ffma_tflops": p_ffma, "mufu_gops": p_mufu, "sm_count": pk["sm_count"],
                                  "hbm_gbs": hbm, "bf16_tflops": bf16_peak}
        phases = {k: st[k] for k in ("ms_generate", "ms_sort", "ms_eval_fp32", "ms_eval_bf16", "ms_shade",
                                     "ms_total")}
        counts = {k: st[k] for k in ("rounds", "rays", "hits", "samples_fp32", "samples_bf16", "samples_tail")}
        accuracy = None
        if precision == kns.KNS_BF16 and fp32 is not None and not args.no_accuracy:
            occ = O.occupancy(desc, w) if desc.occ_res else None
            # both sides must use the same occupancy mask: render the sampled comparison on a grid loaded
            # with the oracle's mask (the timed grid built its mask on the device)
            g2 = kns.Grid.load(ctx, desc, w, occ)
            o_bf = {k: v.cpu().numpy() for k, v in kns.render(ctx, g2, cams, W, H, ms, eps, precision=kns.KNS_BF16).items()}
            o_fp = {k: v.cpu().numpy() for k, v in kns.render(ctx, g2, cams, W, H, ms, eps).items()}
            ctx.sync()
            g2.free()
            accuracy = bf16_accuracy(O, desc, w, occ, cams, W, H, ms, eps, o_bf, o_fp)
        serving = None
        if args.serving and precision == kns.KNS_BF16 and world == 1:
            serving = serving_run(kns, S, (desc, w), args.serving_rates, args.serving_seconds)
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            v, n, s, cores = oracle_rate(desc, w, cams, W, H, ms, eps, args.cpu_seconds)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d rays drawn (seeded, with replacement) from the %d rays of the workload "
                             "(%.1f s of FP64 oracle work)" % (n, n_rays, s)}
        if precision == kns.KNS_BF16:
            launches = 9  # gen, persistent trace, tail, hit count/scan/scatter, shade, refine (+ hit-sort memset)
            launch_src = ("fixed sequence of a BF16 render: ray generation, the persistent trace (every round in one "
                          "cooperative launch), the one-warp-per-ray tail, hit count/scan/scatter, shading, FP32 "
                          "refinement")
        else:
            launches = 4 + st["rounds"] * 5
            launch_src = ("library round counter: gen + rounds x (scan part, scan final, scatter, eval, tail) + "
                          "(rounds - 1) advance + hit sort (3) + shade")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == kns.KNS_FP32 else "bf16",
                "data": "synthetic",
                "config": dict(workload_config(args.workload, desc, cams, W, H, ms, eps, args.precision),
                               parallelism="replicas" if world > 1 else "single GPU",
                               gpu="%s, %d SMs" % (props.name, props.multi_processor_count)),
                "fp32": fp32, "speedup_vs_fp32": (value / fp32["value"]) if fp32 else None,
                "bf16_accuracy_vs_oracle": accuracy,
                "roofline": roof, "cpu_baseline": cpu, "phases_ms_per_render": phases, "counts_per_render": counts,
                "rounds_live": [r["live"] for r in trace][:40],
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "serving": serving,
                "clocks": clock_info, "gpu_launches": args.steps * launches, "tuning": tuning,
                "launch_count_source": launch_src,
                "step_ms_min": min(times), "step_ms_median": statistics.median(times)}
        print(json.dumps(line), flush=True)
    grid.free()
    ctx.close()


# ---------------------------------------------------------------- path tracing
PT_METRIC = "Mpaths/s Lambertian path tracing (sphere-traced bounces)"
PT_WORKLOAD = dict(grid="c2", n_cams=1, W=800, H=800, spp=16, max_depth=4, offset=1e-2, max_steps=128, eps=1e-4)


def oracle_pt_rate(desc, w, occ, cams, seconds: float, seed: int = 0):
    """Times the FP64 oracle's path tracer (as it stands) on seeded random pixels of the workload."""
    import oracle as O
    wl = PT_WORKLOAD
    rng = np.random.default_rng(seed)
    n_pix = wl["n_cams"] * wl["W"] * wl["H"]
    done, elapsed, batch = 0, 0.0, 64
    while elapsed < seconds:
        sel = np.sort(rng.integers(0, n_pix, batch))
        t0 = time.perf_counter()
        O.path_trace(desc, w, occ, cams, wl["W"], wl["H"], wl["spp"], wl["max_depth"], wl["max_steps"], wl["eps"],
                     wl["offset"], seed, (1.0, 1.0, 1.0), (0.5, 0.7, 1.0), sel=sel)
        dt = time.perf_counter() - t0
        elapsed += dt
        done += batch * wl["spp"]
        if dt < seconds / 8:
            batch *= 2
    return done / elapsed / 1e6, done, elapsed, O.num_threads()


def run_pt_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    from paper_2206_10885_gb300 import synth as S
    wl = PT_WORKLOAD
    desc = S.config_desc(wl["grid"])
    w = S.sal_sphere_grid(desc, seed=0)
    occ = O.occupancy(desc, w)
    cams = S.orbit_cameras(wl["n_cams"], wl["W"], wl["H"], seed=1)
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_pt_rate(desc, w, occ, cams, 0.2)
    total, total_s, cores = 0, 0.0, 1
    for k in range(args.steps):
        v, n, s, cores = oracle_pt_rate(desc, w, occ, cams, per_step, seed=k + 1)
        total += n
        total_s += s
    value = total / total_s / 1e6
    n_paths = wl["n_cams"] * wl["W"] * wl["H"] * wl["spp"]
    line = {"impl": "reference", "metric": PT_METRIC, "value": value, "unit": "Mpaths/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_paths / (value * 1e6),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "pt (FP64 oracle)", "paths_per_step": n_paths},
            "cpu_baseline": {"value": value, "unit": "Mpaths/s", "cores": cores, "kind": "oracle",
                             "sample": "%d paths of seeded random pixels over %d steps (%.1f s)"
                                       % (total, args.steps, total_s)},
            "e2e": {"value": value, "unit": "Mpaths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_pt(args, rank, world, local_rank):
    import torch

    import paper_2206_10885_gb300 as kns
    from paper_2206_10885_gb300 import build as kbuild
    from paper_2206_10885_gb300 import synth as S
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2206_10885_gb300", "libkns.so")):
        kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = PT_WORKLOAD
    desc = S.config_desc(wl["grid"])
    w = S.sal_sphere_grid(desc, seed=0)
    cams = S.orbit_cameras(wl["n_cams"], wl["W"], wl["H"], seed=1)
    ctx = kns.Context(local_rank)
    grid = kns.Grid.load(ctx, desc, w)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    n_paths = wl["n_cams"] * wl["W"] * wl["H"] * wl["spp"]

    def step(k):
        return kns.path_trace(ctx, grid, cams, wl["W"], wl["H"], spp=wl["spp"], max_depth=wl["max_depth"], seed=k,
                              offset=wl["offset"], max_steps=wl["max_steps"], eps=wl["eps"])

    for k in range(max(3, args.warmup)):
        step(k)
    torch.cuda.synchronize()
    st = ctx.render_stats()
    clocks = ClockSampler(local_rank).start() if rank == 0 else None
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record(stream)
        step(100 + k)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in evs]
    clock_info = clocks.stop() if clocks else None
    total_ms, = max_over_ranks([sum(times)], dev, world)
    value = whole_job_rate(n_paths, world, args.steps, total_ms)
    # e2e: cameras from host memory every step, the image read back to pinned host memory
    host = torch.empty((wl["n_cams"] * wl["W"] * wl["H"], 3), dtype=torch.float32, pin_memory=True)
    t0 = time.perf_counter()
    for k in range(args.steps):
        host.copy_(step(200 + k), non_blocking=True)
        stream.synchronize()
    e2e_s, = max_over_ranks([time.perf_counter() - t0], dev, world)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            import oracle as O
            v, n, s_, cores = oracle_pt_rate(desc, w, O.occupancy(desc, w), cams, args.cpu_seconds)
            cpu = {"value": v, "unit": "Mpaths/s", "cores": cores, "kind": "oracle",
                   "sample": "%d paths of seeded random pixels (%.1f s of FP64 oracle work)" % (n, s_)}
        line = {"metric": PT_METRIC, "value": value, "unit": "Mpaths/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "pt: Lambertian path tracing of the 16^3 Kilo-grid (3 hidden x 32), 1 orbit "
                                       "camera at 800x800, 16 paths per pixel, up to 4 traces per path, sky "
                                       "gradient; every trace is a wavefront sphere trace (max 128 steps, eps 1e-4)",
                           "paths_per_step": n_paths, "l2": "flushed between steps (512 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "counts_last_warmup_step": {k: st[k] for k in ("rays", "hits", "samples_fp32")},
                "cpu_baseline": cpu,
                "e2e": {"value": whole_job_rate(n_paths, world, args.steps, e2e_s * 1e3), "unit": "Mpaths/s",
                        "h2d_bytes_per_step": int(cams.nbytes), "d2h_bytes_per_step": int(host.numel() * 4)},
                "clocks": clock_info, "step_ms_min": min(times), "step_ms_median": statistics.median(times)}
        print(json.dumps(line), flush=True)
    grid.free()
    ctx.close()


# ---------------------------------------------------------------- training step
TRAIN_METRIC = "Mrays/s through the NeuS training step (loss + hand-written backward)"


def train_macs(desc):
    """Algorithmic multiply-adds per record (biases and activations not counted).

    fwd_d: d of the SDF MLP (coarse samples, difference points); fwd_full: d and z plus the colour MLP
    (sample centres); bwd_d / bwd_full: the backward pass of a record, input gradients through the
    layers plus the weight gradient (one multiply-add per weight), excluding any recomputation of the
    forward pass."""
    IN = 3 + 6 * desc.pe_pos_L
    Wd, Hd = desc.sdf_width, desc.sdf_hidden
    fwd_d = IN * Wd + (Hd - 1) * Wd * Wd + Wd
    sdf_full = IN * Wd + (Hd - 1) * Wd * Wd + Wd * (1 + desc.feat_dim)
    cin = desc.feat_dim + 3 + 3 + 6 * desc.pe_dir_L
    col = cin * desc.col_width + desc.col_width * 3
    bwd_d = (Wd + (Hd - 1) * Wd * Wd) + fwd_d
    col_back_in = desc.col_width * 3 + (desc.feat_dim + 3) * desc.col_width
    bwd_full = (Wd * (1 + desc.feat_dim) + (Hd - 1) * Wd * Wd) + sdf_full + col_back_in + col
    return {"fwd_d": fwd_d, "fwd_full": sdf_full + col, "bwd_d": bwd_d, "bwd_full": bwd_full}


def train_setup(torch, kns, S, ctx, dev, seed, n_rays=0):
    wl = dict(S.TRAIN_WORKLOAD)
    if n_rays:
        wl.update(n_rays=n_rays, n_eik=max(1, n_rays * wl["n_eik"] // wl["n_rays"]))
    desc = S.config_desc(wl["grid"])
    W, H, n_cams = wl["W"], wl["H"], wl["n_cams"]
    cams = S.orbit_cameras(n_cams, W, H, seed=1)
    tw = S.sal_sphere_grid(desc, seed=wl["target_seed"], perturb_std=wl["target_std"])
    tgrid = kns.Grid.load(ctx, desc, tw)
    img = kns.render(ctx, tgrid, cams, W, H, wl["max_steps"], wl["eps"])["rgb"]
    sel, u_s, u_i, P = S.train_draws(wl["n_rays"], wl["n_strat"], wl["n_imp"], wl["n_eik"], n_cams * W * H, seed)
    o, d = S.pixel_rays(cams, W, H, sel)
    tgt = img[torch.from_numpy(sel).to(dev)].contiguous()
    torch.cuda.synchronize()
    tgrid.free()
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    host = dict(o=o, d=d, target=tgt.cpu().numpy(), u_s=u_s, u_i=u_i, P=P)
    batch = kns.train.TrainBatch(f(o), f(d), tgt, f(u_s), f(u_i), f(P), s=wl["s"], s_up=wl["s_up"], lam=wl["lam"],
                                 h=wl["h"])
    params = f(S.sal_sphere_grid(desc, seed=0))
    return wl, desc, batch, params, host


def train_config(wl, desc, dtype_note):
    return {"workload": "train: NeuS training step on a %d^3 Kilo-grid (SDF MLP %d hidden x %d, softplus beta=%g, "
                        "PE L=%d; colour MLP %d x %d); %d rays x (%d stratified + %d importance) samples, L1 colour "
                        "+ %g x eikonal on %d points, s=%g, s_up=%g, central-difference step h=%g; %s"
                        % (desc.N, desc.sdf_hidden, desc.sdf_width, desc.softplus_beta, desc.pe_pos_L,
                           desc.col_hidden, desc.col_width, wl["n_rays"], wl["n_strat"], wl["n_imp"], wl["lam"],
                           wl["n_eik"], wl["s"], wl["s_up"], wl["h"], dtype_note),
            "rays_per_step": wl["n_rays"], "samples_per_ray": wl["n_strat"] + wl["n_imp"],
            "eikonal_points": wl["n_eik"], "grid": "%d^3" % desc.N,
            "l2": "flushed between steps (512 MiB write outside the timed events); step scratch ~5 GB > L2",
            "inputs": "synthetic: rays at seeded random pixels of 8 orbit cameras at 800x800, targets rendered "
                      "from a perturbed sphere grid (seed 3, std 1e-2), trained weights = SAL grid seed 0"}


def oracle_train_rate(desc, w, host, wl, seconds: float, seed: int = 0):
    """Times the FP64 oracle's loss + gradient (as it stands) on seeded random subsets of the batch."""
    import oracle as O
    rng = np.random.default_rng(seed)
    B, M = wl["n_rays"], wl["n_eik"]
    done, elapsed, n = 0, 0.0, 8
    while elapsed < seconds:
        r = rng.choice(B, n, replace=False)
        m = rng.choice(M, max(1, n * M // B), replace=False)
        args = (wl["s"], wl["s_up"], host["o"][r].astype(np.float64), host["d"][r].astype(np.float64),
                host["target"][r].astype(np.float64), host["u_s"][r].astype(np.float64),
                host["u_i"][r].astype(np.float64), host["P"][m].astype(np.float64), wl["lam"], wl["h"])
        t0 = time.perf_counter()
        O.train_grad(desc, w, *args)
        dt = time.perf_counter() - t0
        elapsed += dt
        done += n
        if dt < seconds / 8:
            n *= 2
    return done / elapsed / 1e6, done, elapsed, O.num_threads()


def oracle_train_inputs(S, wl, desc, n: int = 4096):
    """The first n rays of the training batch (the GPU arm's draws) with targets rendered by the oracle."""
    import oracle as O
    n = min(n, wl["n_rays"])
    cams = S.orbit_cameras(wl["n_cams"], wl["W"], wl["H"], seed=1)
    sel, u_s, u_i, P = S.train_draws(wl["n_rays"], wl["n_strat"], wl["n_imp"], wl["n_eik"],
                                     wl["n_cams"] * wl["W"] * wl["H"], 0)
    o, d = S.pixel_rays(cams, wl["W"], wl["H"], sel[:n])
    tw = S.sal_sphere_grid(desc, seed=wl["target_seed"], perturb_std=wl["target_std"])
    tgt = O.render(desc, tw, None, cams, wl["W"], wl["H"], wl["max_steps"], wl["eps"], sel=sel[:n])["rgb"]
    m = max(1, n * wl["n_eik"] // wl["n_rays"])  # the batch's share of eikonal points
    return dict(o=o, d=d, target=tgt, u_s=u_s[:n], u_i=u_i[:n], P=P[:m]), dict(wl, n_rays=n, n_eik=m)


def run_train_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2206_10885_gb300 import synth as S
    wl = S.TRAIN_WORKLOAD
    desc = S.config_desc(wl["grid"])
    host, wl_sub = oracle_train_inputs(S, wl, desc)
    w = S.sal_sphere_grid(desc, seed=0)
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_train_rate(desc, w, host, wl_sub, 0.2)
    total, total_s, cores = 0, 0.0, 1
    for k in range(args.steps):
        v, n, s, cores = oracle_train_rate(desc, w, host, wl_sub, per_step, seed=k + 1)
        total += n
        total_s += s
    value = total / total_s / 1e6
    line = {"impl": "reference", "metric": TRAIN_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wl["n_rays"] / (value * 1e6),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": train_config(wl, desc, "fp64 oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d seeded random rays of the first 4096 of the batch, with their share of "
                                       "eikonal points, over %d steps (%.1f s)" % (total, args.steps, total_s)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_train(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_2206_10885_gb300 as kns
    from paper_2206_10885_gb300 import build as kbuild
    from paper_2206_10885_gb300 import synth as S

    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2206_10885_gb300", "libkns.so")):
        kbuild.build()
    if world > 1:
        dist.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = kns.Context(local_rank)
    wl, desc, batch, params, host = train_setup(torch, kns, S, ctx, dev, seed=rank, n_rays=args.train_rays)
    stream = torch.cuda.current_stream()
    loss = torch.empty(3, dtype=torch.float32, device=dev)
    grad = torch.empty_like(params)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step():
        kns.train.step(ctx, desc, params, batch, stream=stream, loss_out=loss, grad_out=grad)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # per-phase device time and record counts from a step timed with CUDA events
    batch.timing = True
    step()
    st = kns.train.stats(ctx)
    batch.timing = False
    mac = train_macs(desc)

    clocks = ClockSampler(local_rank).start() if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(times)
    # e2e through the public API: the batch's inputs copied from pinned host memory every step, the
    # loss read back
    pin = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).pin_memory() for k, v in host.items()}
    dev_in = {"o": batch.origins, "d": batch.dirs, "target": batch.target, "u_s": batch.u_strat,
              "u_i": batch.u_imp, "P": batch.eik_points}
    loss_host = torch.empty(3, dtype=torch.float32, pin_memory=True)
    h2d = sum(v.numel() * v.element_size() for v in pin.values())
    d2h = loss_host.numel() * 4
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for k, v in pin.items():
            dev_in[k].copy_(v, non_blocking=True)
        step()
        loss_host.copy_(loss, non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    clock_info = clocks.stop() if clocks else None

    total_ms, e2e_s = max_over_ranks([total_ms, e2e_s], dev, world)
    n_rays = wl["n_rays"]
    value = whole_job_rate(n_rays, world, args.steps, total_ms)
    if rank == 0:
        fp32_peak = ctx.measure_peaks(stream)["ffma_flops"] / 1e12
        flops = 2.0 * st["records_fd"] * mac["bwd_d"]
        kms = st["ms_fd_backward"]
        achieved = flops / (kms * 1e-3) / 1e12 if kms > 0 else 0.0
        roof = {"bound": "alu", "peak": fp32_peak, "unit": "TFLOP/s",
                "kernel": "k_tile_backward (difference points)",
                "peak_source": "measured on this GPU: FFMA micro-kernel (kns_measure_peaks), of measured",
                "achieved": achieved, "frac": achieved / fp32_peak,
                "traffic": profile_traffic("k_tile_backward_fd_train"), "algorithmic_flop_per_launch": flops,
                "kernel_ms_per_launch": kms, "flop_per_record": 2 * mac["bwd_d"],
                "records_per_launch": st["records_fd"],
                "note": "algorithmic work = input gradients + weight gradient; the kernel also recomputes the "
                        "forward pass of each record (%d more FLOP per record), not counted" % (2 * mac["fwd_d"])}
        phases = {k: st[k] for k in st if k.startswith("ms_")}
        counts = {k: st[k] for k in ("rays", "samples_per_ray", "eik_points", "records_coarse", "records_fd",
                                     "records_centre")}
        work = {"fp32_flop_algorithmic": 2.0 * (st["records_coarse"] * mac["fwd_d"] +
                                                st["records_fd"] * (mac["fwd_d"] + mac["bwd_d"]) +
                                                st["records_centre"] * (mac["fwd_full"] + mac["bwd_full"]))}
        work["fp32_tflops_whole_step"] = work["fp32_flop_algorithmic"] / (total_ms / args.steps * 1e-3) / 1e12
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            o_host, wl_sub = oracle_train_inputs(S, wl, desc)
            v, n, s, cores = oracle_train_rate(desc, params.cpu().numpy(), o_host, wl_sub, args.cpu_seconds)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d seeded random rays of the first 4096 of the %d-ray batch with their share of the "
                             "eikonal points (%.1f s of FP64 oracle loss + gradient)" % (n, n_rays, s)}
        line = {"metric": TRAIN_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(train_config(wl, desc, "fp32"),
                               parallelism="replicas" if world > 1 else "single GPU"),
                "roofline": roof, "cpu_baseline": cpu, "phases_ms_per_step": phases, "counts_per_step": counts,
                "work_per_step": work,
                "e2e": {"value": whole_job_rate(n_rays, world, args.steps, e2e_s * 1e3), "unit": UNIT,
                        "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
                "clocks": clock_info, "gpu_launches": args.steps * 17,
                "launch_count_source": "fixed kernel sequence of kns_train_step: coarse hist/scan/scatter/eval, "
                                       "importance, fine hist/scan/scatter, difference and centre forward, "
                                       "composite, eikonal, finalize, composite and eikonal upstream, centre and "
                                       "difference backward (memsets and copies not counted)",
                "step_ms_min": min(times), "step_ms_median": statistics.median(times),
                "final_loss": [float(x) for x in loss.cpu()]}
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload == "train":
            run_train_reference(args, rank, world)
        elif args.workload == "pt":
            run_pt_reference(args, rank, world)
        else:
            run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "train":
        run_train(args, rank, world, local_rank)
    elif args.workload == "pt":
        run_pt(args, rank, world, local_rank)
    else:
        run_kns(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
