"""Continuous-batching render server over resident Kilo-grids.

Requests (grid, camera, W, H) arrive at any time.  Worker slots each own a kns context (so their
device scratch is separate), a CUDA stream and a host thread, so batches on different slots are
issued and run concurrently on the GPU.  Grids of one shape (the same descriptor) are loaded as one
stack (kns_load_grid_stack), so a batch can hold requests for any of them: a free slot takes the
stack of the oldest waiting request and batches every admitted request for any grid of that stack
(up to max_batch_rays) into one kns_render_views call, each view naming its grid: one launch
sequence renders all of their rays, whatever their grids and resolutions.  A request is
admitted once its output buffers fit in the HBM budget next to the requests in flight; requests
that arrive while others are on the GPU join the next batch a slot forms.  Latency is measured
from a request's (scheduled) arrival to the end of its batch on the slot's stream.

CLI (one GPU): python -m paper_2206_10885_gb300.serve --rates 50 100 200 400 --seconds 4
prints one JSON line per arrival rate with Mrays/s and p50/p99 frame latency.
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import gc
import json
import math
import threading
import time

import numpy as np

from . import KNS_BF16, KNS_FP32, Context, Grid, alloc_frame, render_views
from . import synth as S

BYTES_PER_PIXEL = 12 + 4 + 12 + 4 + 4 + 1  # rgb, depth, normal, cell, steps, hit


def desc_key(desc) -> tuple:
    """Grids whose descriptors give equal keys can share one stack."""
    return tuple([int(getattr(desc, k)) for k in ("N", "pe_pos_L", "pe_dir_L", "sdf_hidden", "sdf_width", "feat_dim",
                                                   "col_hidden", "col_width", "col_use_x", "occ_res")]
                 + [float(desc.softplus_beta)] + [float(x) for x in desc.bbox_min] + [float(x) for x in desc.bbox_max])


@dataclasses.dataclass
class Request:
    rid: int
    grid: str
    cam: np.ndarray
    W: int
    H: int
    arrival: float = 0.0      # seconds (server clock)
    taken: float = -1.0       # when a slot took it into a batch
    done: float = -1.0
    batch: int = -1           # the batch that rendered it
    out: dict = None

    @property
    def rays(self) -> int:
        return self.W * self.H

    @property
    def bytes(self) -> int:
        return self.rays * BYTES_PER_PIXEL


class _Slot:
    def __init__(self, device: int):
        import torch
        self.ctx = Context(device)
        self.stream = torch.cuda.Stream(device=device)
        self.thread = None


class RenderServer:
    """Resident grids + K worker slots + admission by HBM budget + continuous batching.

    Each slot runs a worker thread: it takes a batch (all admitted requests for the grids of the oldest
    one's stack, up to max_batch_rays), renders it with one kns_render_views call on the slot's own
    context and stream, waits for the stream and stamps the requests' completion time.  Host waits
    inside a render (FP32 renders poll the live-ray count between rounds; BF16 renders run their
    rounds in one persistent launch) happen in that thread, so batches on different slots are
    issued and executed concurrently.
    """

    def __init__(self, grids: dict, device: int = 0, slots: int = 3, budget_bytes: int = 8 << 30,
                 max_batch_rays: int = 8 << 20, max_steps: int = 128, eps: float = 1e-4,
                 precision: int = KNS_FP32, tuning=None, stack: bool = True):
        self.device = device
        self.slots = [_Slot(device) for _ in range(slots)]
        # grids: name -> (desc, weights[, occupancy words]).  Grids with equal descriptors share one stack;
        # a stack lives in device memory and is usable from every context on the device
        self.grids = {}       # name -> (stack key, index of the grid in its stack)
        self.stacks = {}      # stack key -> Grid
        self.group_of = {}    # name -> stack key
        loader = self.slots[0].ctx
        groups = collections.OrderedDict()
        for name, spec in grids.items():  # stack=False: every grid a stack of its own (batches of one grid)
            groups.setdefault(desc_key(spec[0]) if stack else (name,), []).append((name, spec))
        for key, members in groups.items():
            desc = members[0][1][0]
            occ = [m[1][2] for m in members] if all(len(m[1]) > 2 and m[1][2] is not None for m in members) else None
            if len(members) == 1:
                self.stacks[key] = Grid.load(loader, desc, members[0][1][1], occ[0] if occ else None)
            else:
                self.stacks[key] = Grid.load_stack(loader, desc, [m[1][1] for m in members], occ)
            for k, (name, _) in enumerate(members):
                self.grids[name] = (key, k)
                self.group_of[name] = key
        self.budget = budget_bytes
        self.max_batch_rays = max_batch_rays
        self.max_steps, self.eps, self.precision, self.tuning = max_steps, eps, precision, tuning
        self.pending = collections.deque()
        self.in_flight_bytes = 0
        self.in_flight = 0
        self.completed = []
        self.cv = threading.Condition()
        self.t0 = time.perf_counter()
        self.batches = 0
        self.mixed_batches = 0  # batches holding requests for more than one grid
        self.running = True
        self.error = None
        self._warm()
        for sl in self.slots:
            sl.thread = threading.Thread(target=self._worker, args=(sl,), daemon=True)
            sl.thread.start()

    def _warm(self) -> None:
        """Each slot renders, on each stack, one batch as large as a batch can be (max_batch_rays rays in
        large views, plus 128 one-pixel views for the view table), so that its context's scratch already
        holds any batch it will form: no batch allocates device memory, or waits for it, while serving."""
        import torch
        W = 2048
        H = max(1, min(2048, -(-self.max_batch_rays // W)))
        n = max(1, -(-self.max_batch_rays // (W * H)))
        cam = S.orbit_cameras(1, W, H, seed=0)[0]
        views = [(cam, W, H, 0)] * n + [(cam, 1, 1, 0)] * 128
        for sl in self.slots:
            for stack in self.stacks.values():
                with torch.cuda.stream(sl.stream):
                    render_views(sl.ctx, stack, views, self.max_steps, self.eps, precision=self.precision,
                                 stream=sl.stream, tuning=self.tuning)
                sl.stream.synchronize()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request, arrival: float = None) -> None:
        with self.cv:
            req.arrival = self.now() if arrival is None else arrival
            self.pending.append(req)
            self.cv.notify()

    def _take_batch(self):
        """Admitted requests for the grids of the oldest request's stack (caller holds the lock).
        Returns (stack key, requests)."""
        if not self.pending:
            return None, []
        group = getattr(self, "group_of", {})
        key = group.get(self.pending[0].grid, self.pending[0].grid)
        take, rays, keep = [], 0, collections.deque()
        while self.pending:
            r = self.pending.popleft()
            fits = self.in_flight_bytes + r.bytes <= self.budget or (not take and self.in_flight_bytes == 0)
            if group.get(r.grid, r.grid) == key and fits and (not take or rays + r.rays <= self.max_batch_rays):
                take.append(r)
                rays += r.rays
                self.in_flight_bytes += r.bytes
            else:
                keep.append(r)
        self.pending = keep
        if take:
            self.in_flight += 1
            self.batches += 1
            now = self.now() if hasattr(self, "t0") else 0.0
            for r in take:
                r.batch, r.taken = self.batches, now
            if len({r.grid for r in take}) > 1:
                self.mixed_batches += 1
        return key, take

    def _worker(self, slot: _Slot) -> None:
        import torch
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while self.running and not self.pending:
                    self.cv.wait(0.01)
                if not self.running and not self.pending:
                    return
                key, take = self._take_batch()
            if not take:
                time.sleep(20e-6)
                continue
            try:
                with torch.cuda.stream(slot.stream):
                    outs = [alloc_frame(r.rays, "cuda:%d" % self.device) for r in take]
                    views = [(r.cam, r.W, r.H, self.grids[r.grid][1]) for r in take]
                    tensors = render_views(slot.ctx, self.stacks[key], views, self.max_steps, self.eps,
                                           precision=self.precision, stream=slot.stream, outs=outs,
                                           tuning=self.tuning)
                slot.stream.synchronize()
            except Exception as e:  # surfaced by drain()
                self.error = e
                tensors = [None] * len(take)
            t = self.now()
            with self.cv:
                for r, out in zip(take, tensors):
                    r.out, r.done = out, t
                    self.in_flight_bytes -= r.bytes
                    self.completed.append(r)
                self.in_flight -= 1
                self.cv.notify_all()

    def drain(self, timeout_s: float = 120.0) -> None:
        end = time.perf_counter() + timeout_s
        with self.cv:
            while (self.pending or self.in_flight) and time.perf_counter() < end:
                self.cv.wait(0.01)
        if self.error is not None:
            raise self.error

    def close(self) -> None:
        self.drain()
        with self.cv:
            self.running = False
            self.cv.notify_all()
        for sl in self.slots:
            sl.thread.join(timeout=10)
        for g in self.stacks.values():
            g.free()
        for sl in self.slots:
            sl.ctx.close()


def poisson_stream(n: int, rate: float, seed: int, grids, resolutions, start_id: int = 0):
    """n requests: exponential inter-arrival times (rate per second), uniform grid and resolution."""
    u = S.uniform(S.stream_key(seed, 6), 4 * n).reshape(n, 4)
    t, out = 0.0, []
    for i in range(n):
        t += -math.log(1.0 - u[i, 0]) / rate
        W, H = resolutions[int(u[i, 1] * len(resolutions)) % len(resolutions)]
        gname = grids[int(u[i, 2] * len(grids)) % len(grids)]
        cam = S.orbit_cameras(1, W, H, seed=seed * 100003 + i)[0]
        out.append((t, Request(start_id + i, gname, cam, W, H)))
    return out


def run_stream(server: RenderServer, stream) -> dict:
    """Submits (arrival offset, request) pairs at their arrival times, waits for all; returns stats.
    Python's cyclic garbage collector is paused meanwhile: a collection holds the interpreter lock for
    tens of milliseconds and would delay the submissions and the workers alike."""
    gc.collect()
    gc.disable()
    try:
        return _run_stream(server, stream)
    finally:
        gc.enable()


def _run_stream(server: RenderServer, stream) -> dict:
    server.t0 = time.perf_counter()
    with server.cv:
        server.completed.clear()
        server.batches = 0
        server.mixed_batches = 0
    for t_arr, req in stream:
        delay = t_arr - server.now()
        if delay > 0:
            time.sleep(delay)
        server.submit(req, arrival=t_arr)
    server.drain()
    done = [r for r in server.completed if r.rid >= 0]
    lat = np.array([(r.done - r.arrival) * 1e3 for r in done])
    rays = sum(r.rays for r in done)
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"requests": len(done), "rays": rays, "seconds": span, "mrays_per_s": rays / span / 1e6,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "batches": server.batches, "mixed_batches": server.mixed_batches}


RES_MIX = [(256, 256), (512, 512), (800, 800), (1920, 1080)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", type=float, nargs="+", default=[50, 100, 200, 400])
    ap.add_argument("--seconds", type=float, default=4.0)
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-stack", action="store_true", help="batches of one grid each (no grid stacks)")
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    grids = {}
    for k, (gname, seed) in enumerate([("c3s", 0), ("c3s", 1), ("c3l", 0), ("c3l", 1)]):
        desc = S.config_desc(gname)
        grids["%s-%d" % (gname, seed)] = (desc, S.sal_sphere_grid(desc, seed=seed))
    prec = KNS_BF16 if args.precision == "bf16" else KNS_FP32
    server = RenderServer(grids, slots=args.slots, precision=prec, stack=not args.no_stack)
    names = list(grids)
    # warm every slot on every grid with the largest resolution (grows each context's scratch once)
    warm = [Request(-1 - k, names[k % len(names)], S.orbit_cameras(1, 1920, 1080, seed=k)[0], 1920, 1080)
            for k in range(len(names) * args.slots)]
    for r in warm:
        server.submit(r)
    server.drain()
    for rate in args.rates:
        n = max(8, int(rate * args.seconds))
        stream = poisson_stream(n, rate, seed=int(rate), grids=names, resolutions=RES_MIX)
        res = run_stream(server, stream)
        res.update({"rate_per_s": rate, "precision": args.precision, "slots": args.slots, "stack": not args.no_stack,
                    "grids": "2 x 16^3/w32 + 2 x 32^3/w64", "resolutions": "256^2, 512^2, 800^2, 1920x1080"})
        print(json.dumps(res), flush=True)
    server.close()


if __name__ == "__main__":
    main()
