"""Render server with continuous batching over resident VDB scenes.

Every scene's grid, blob field and lattice parameters stay on the device.
Render requests (a scene, a camera's rays) arrive at any time and wait in a
FIFO queue.  The server has a fixed number of slots; each slot is a worker
thread with its own CUDA stream.  A request is admitted as soon as a slot is
free and its estimated device memory fits the budget, so requests that arrive
while others are running join them on the GPU instead of waiting for a batch
boundary.  Each admission point takes every queued request that fits, in
order (one "tick").

Three executor modes:
  "samples"  the frame goes through the sample buffers (traversal, then
             compositing), as the paper's renderer does.  The estimate is rays
             x (rays, offsets, colours, traversal scratch) plus samples x 12
             bytes, with samples per ray taken from a per-scene decaying
             maximum over completed requests, plus headroom.  If a frame needs
             more samples than reserved, the sampler reports the exact total
             and the slot re-runs at that size.
  "batched"  as "samples", but a slot takes every request that is ready when
             it frees up (up to `max_batch`, one admission tick's worth) and
             samples all of them in ONE batched launch (hdda_batch: the
             requests' rays are cut into 32-ray tiles that persistent warps
             take from one counter, across requests and scenes), then
             composites each frame; a frame that outgrew its reservation is
             re-run alone at the exact size.
  "render"   the render-only path (hdda_render): no sample buffers, so a
             request costs a fixed number of bytes per ray, never re-runs, and
             the library does not wait for the device before the frame's copy.

Per request, in the slot's stream:
  1. the rays are copied to the device;
  2. "samples": the HDDA sampler walks them (walk, scan and emit, one host
     read of the total) and the compositor renders the frame; "render": the
     walk and the run-level compositor render it;
  3. the frame is copied back to pinned host memory.

Latency runs from arrival to the frame in host memory.  The library calls
release the GIL, so the slots' GPU work overlaps.

The admission policy (`Admission`) is plain Python and is tested without a
GPU.
"""
from __future__ import annotations

import collections
import statistics
import threading
import time
from dataclasses import dataclass, field

BYTES_PER_RAY = 24 + 8 + 16 + 4 + 1 + 128 + 24  # rays, offsets, rgba, counts, runs, slack
BYTES_PER_SAMPLE = 12
BYTES_PER_RAY_RENDER = 24 + 16 + 4 + 1 + 128 + 8  # rays, rgba, counts, runs, slack


@dataclass
class Request:
    rid: int
    scene: int
    rays_o: object             # host float32 [n, 3] (pinned for a real server)
    rays_d: object
    arrival: float = 0.0
    admitted: float = 0.0
    done: float = 0.0
    reserved: int = 0
    samples: int = 0
    retries: int = 0
    rgba: object = None        # host float32 [n, 4]
    error: str | None = None
    width: int = 0             # image width when the rays are an image's pixels row by row

    @property
    def n_rays(self) -> int:
        return int(self.rays_o.shape[0])

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Admission:
    """FIFO admission against a device-memory budget and a slot count."""

    def __init__(self, budget_bytes: int, slots: int, samples_per_ray_hint: float = 64.0,
                 headroom: float = 1.5, bytes_per_ray: int = BYTES_PER_RAY,
                 bytes_per_sample: int = BYTES_PER_SAMPLE):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.bytes_per_ray = bytes_per_ray
        self.bytes_per_sample = bytes_per_sample
        self.in_use = 0
        self.busy = 0
        self.headroom = headroom
        self.hint = samples_per_ray_hint
        self.spr: dict[int, float] = {}
        self.queue: collections.deque = collections.deque()

    def estimate_samples(self, req: Request) -> int:
        if not self.bytes_per_sample:
            return 0
        return int(req.n_rays * self.spr.get(req.scene, self.hint) * self.headroom) + 1024

    def estimate_bytes(self, req: Request, samples: int | None = None) -> int:
        s = self.estimate_samples(req) if samples is None else samples
        return req.n_rays * self.bytes_per_ray + s * self.bytes_per_sample

    def push(self, req: Request) -> None:
        self.queue.append(req)

    def pop_admissible(self) -> list[Request]:
        """Every queued request that fits now, in order, stopping at the first that does
        not (no overtaking, so large frames cannot starve).  A request larger than the
        whole budget is admitted alone when nothing else runs."""
        out = []
        while self.queue and self.busy < self.slots:
            req = self.queue[0]
            need = self.estimate_bytes(req)
            if self.in_use + need > self.budget and not (self.busy == 0 and not out):
                break
            self.queue.popleft()
            req.reserved = need
            self.in_use += need
            self.busy += 1
            out.append(req)
        return out

    def resize(self, req: Request, samples: int) -> None:
        """A frame needed `samples`: its reservation becomes exact."""
        need = self.estimate_bytes(req, samples)
        self.in_use += need - req.reserved
        req.reserved = need

    def release(self, req: Request) -> None:
        self.in_use -= req.reserved
        self.busy -= 1
        if req.samples and req.n_rays:
            # a decaying maximum: follows the heaviest recent views of the scene
            spr = req.samples / req.n_rays
            old = self.spr.get(req.scene)
            self.spr[req.scene] = spr if old is None else max(spr, 0.97 * old)


class RenderServer:
    """Continuous-batching server.  `executor(slot, req)` renders one request in the
    slot's stream and fills req.rgba / req.samples (GpuExecutor below); it may raise
    NeedMore(samples) to ask for an exact re-run."""

    def __init__(self, executor, slots: int, budget_bytes: int, samples_per_ray_hint: float = 64.0,
                 max_batch: int = 8):
        self.exec = executor
        self.max_batch = max_batch if getattr(executor, "batched", False) else 1
        self.adm = Admission(budget_bytes, slots, samples_per_ray_hint,
                             bytes_per_ray=getattr(executor, "bytes_per_ray", BYTES_PER_RAY),
                             bytes_per_sample=getattr(executor, "bytes_per_sample",
                                                      BYTES_PER_SAMPLE))
        self.cv = threading.Condition()
        self.stopping = False
        self.completed: list[Request] = []
        self.ticks = 0
        self.max_concurrent = 0
        self.ready: collections.deque = collections.deque()
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(slots)]
        for t in self.threads:
            t.start()

    def submit(self, req: Request) -> None:
        with self.cv:
            if not req.arrival:
                req.arrival = time.perf_counter()
            self.adm.push(req)
            self._tick()
            self.cv.notify_all()

    def _tick(self) -> None:
        got = self.adm.pop_admissible()
        if got:
            self.ticks += 1
            now = time.perf_counter()
            for r in got:
                r.admitted = now
            self.ready.extend(got)
            self.max_concurrent = max(self.max_concurrent, self.adm.busy)

    def _worker(self, slot: int) -> None:
        while True:
            with self.cv:
                while not self.ready and not self.stopping:
                    self.cv.wait()
                if self.stopping and not self.ready:
                    return
                group = [self.ready.popleft() for _ in range(min(len(self.ready), self.max_batch))]
            rerun = group
            if self.max_batch > 1:
                try:
                    rerun = [r for r, samples in self.exec.batch_call(slot, group)]
                except Exception as e:  # the group fails, the server goes on
                    for r in group:
                        r.error = repr(e)
                    rerun = []
                for r in rerun:  # frames that outgrew their reservation, alone at the exact size
                    r.retries += 1
                with self.cv:
                    for r in rerun:
                        self.adm.resize(r, r.samples)
            for req in rerun:
                self._run_one(slot, req)
            now = time.perf_counter()
            with self.cv:
                for req in group:
                    req.done = now if req.done == 0.0 else req.done
                    self.adm.release(req)
                    self.completed.append(req)
                self._tick()
                self.cv.notify_all()

    def _run_one(self, slot: int, req: Request) -> None:
        while True:
            try:
                self.exec(slot, req, req.reserved)
                break
            except NeedMore as more:
                req.retries += 1
                with self.cv:
                    self.adm.resize(req, more.samples)
            except Exception as e:  # the request fails, the server goes on
                req.error = repr(e)
                break
        req.done = time.perf_counter()

    def drain(self, timeout: float = 120.0) -> None:
        t_end = time.perf_counter() + timeout
        with self.cv:
            while (self.adm.queue or self.adm.busy or self.ready) and time.perf_counter() < t_end:
                self.cv.wait(timeout=0.05)

    def close(self) -> None:
        self.drain()
        with self.cv:
            self.stopping = True
            self.cv.notify_all()
        for t in self.threads:
            t.join(timeout=10)


class NeedMore(Exception):
    def __init__(self, samples: int):
        super().__init__(f"needs {samples} samples")
        self.samples = samples


class GpuExecutor:
    """Renders requests on the GPU: resident scenes, one CUDA stream per slot.
    mode "samples" (sample buffers, then compositing) or "render" (hdda_render)."""

    def __init__(self, scene_list, slots: int, mode: str = "samples"):
        import torch
        from . import hdda
        if mode not in ("samples", "batched", "render"):
            raise ValueError(f"unknown mode {mode!r}")
        self.mode = mode
        self.batched = mode == "batched"
        self.bytes_per_ray = BYTES_PER_RAY if mode != "render" else BYTES_PER_RAY_RENDER
        self.bytes_per_sample = BYTES_PER_SAMPLE if mode != "render" else 0
        self.torch = torch
        self.hdda = hdda
        self.grids, self.fields, self.params = [], [], []
        for sc in scene_list:
            self.grids.append(hdda.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs))
            self.fields.append(torch.from_numpy(sc.field).cuda())
            p = sc.params
            self.params.append(hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step,
                                                p.max_steps))
        torch.cuda.synchronize()
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.status = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in range(slots)]
        self.status_host = [torch.zeros(1, dtype=torch.int32, pin_memory=True)
                            for _ in range(slots)]

    def _params(self, req: Request):
        """The scene's parameters, with the request's image width as the ray-order hint."""
        base = self.params[req.scene]
        if req.width <= 0:
            return base
        prm = type(base).from_buffer_copy(base)
        prm.image_width = req.width
        return prm

    def warm(self) -> None:
        """First use of each scene's lattice synchronises; do it before serving."""
        torch, hdda = self.torch, self.hdda
        for g, prm in zip(self.grids, self.params):
            o = torch.zeros((1, 3), device="cuda")
            hdda.traverse_hdda(o, o + 1.0, g, prm, count_only=True)

    def __call__(self, slot: int, req: Request, reserved_bytes: int) -> None:
        if self.mode == "render":
            return self._render(slot, req)
        torch, hdda = self.torch, self.hdda
        s = self.streams[slot]
        n = req.n_rays
        cap = max(1, (reserved_bytes - n * BYTES_PER_RAY) // BYTES_PER_SAMPLE)
        with torch.cuda.stream(s):
            o = req.rays_o.to("cuda", non_blocking=True)
            d = req.rays_d.to("cuda", non_blocking=True)
            out = hdda.alloc_samples(n, cap)
            g, prm, fld = self.grids[req.scene], self._params(req), self.fields[req.scene]
            try:
                smp = hdda.traverse_hdda(o, d, g, prm, out=out, stream=s)
            except hdda.HddaError as e:
                if e.code == hdda.ERR_CAPACITY:
                    raise NeedMore(out.total) from None
                raise
            rgba = hdda.composite(o, d, smp, fld, stream=s)
            host = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
            host.copy_(rgba, non_blocking=True)
            s.synchronize()
        req.samples = smp.total
        req.rgba = host

    def batch_call(self, slot: int, reqs: list) -> list:
        """Samples every request of the group in one batched launch on the slot's stream,
        then composites each frame.  Returns [(request, samples)] for the frames whose
        samples did not fit their reservation (req.samples holds the exact count)."""
        torch, hdda = self.torch, self.hdda
        s = self.streams[slot]
        with torch.cuda.stream(s):
            jobs = []
            for req in reqs:
                n = req.n_rays
                cap = max(1, (req.reserved - n * BYTES_PER_RAY) // BYTES_PER_SAMPLE)
                jobs.append(dict(rays_o=req.rays_o.to("cuda", non_blocking=True),
                                 rays_d=req.rays_d.to("cuda", non_blocking=True),
                                 grid=self.grids[req.scene], params=self.params[req.scene],
                                 out=hdda.alloc_samples(n, cap)))
            b = hdda.Batch(jobs, use_graph=False, stream=s)
            try:
                b.launch(stream=s)
                totals, status = b.results(stream=s, check=False)
            finally:
                b.free()
            over, hosts = [], []
            for req, jb, tot, st in zip(reqs, jobs, totals, status):
                req.samples = tot
                if st != hdda.OK:
                    over.append((req, tot))
                    hosts.append(None)
                    continue
                rgba = hdda.composite(jb["rays_o"], jb["rays_d"], jb["out"],
                                      self.fields[req.scene], stream=s)
                host = torch.empty((req.n_rays, 4), dtype=torch.float32, pin_memory=True)
                host.copy_(rgba, non_blocking=True)
                hosts.append(host)
            s.synchronize()
        for req, host in zip(reqs, hosts):
            if host is not None:
                req.rgba = host
        return over

    def _render(self, slot: int, req: Request) -> None:
        torch, hdda = self.torch, self.hdda
        s = self.streams[slot]
        n = req.n_rays
        st = self.status[slot]
        with torch.cuda.stream(s):
            o = req.rays_o.to("cuda", non_blocking=True)
            d = req.rays_d.to("cuda", non_blocking=True)
            st.zero_()
            g, prm, fld = self.grids[req.scene], self._params(req), self.fields[req.scene]
            rgba = hdda.render(o, d, g, prm, fld, status=st, stream=s)
            host = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
            host.copy_(rgba, non_blocking=True)
            sh = self.status_host[slot]
            sh.copy_(st, non_blocking=True)   # read with the frame: one wait per request
            s.synchronize()
        if int(sh[0]) != 0:
            raise RuntimeError(f"hdda_render raised device status {int(sh[0])}")
        req.rgba = host


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = (len(xs) - 1) * q
    lo, hi = int(k), min(int(k) + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def summary(reqs: list[Request], wall: float) -> dict:
    lat = [r.latency * 1e3 for r in reqs if r.error is None]
    rays = sum(r.n_rays for r in reqs if r.error is None)
    return {"requests": len(reqs), "errors": sum(r.error is not None for r in reqs),
            "p50_ms": round(percentile(lat, 0.5), 3), "p99_ms": round(percentile(lat, 0.99), 3),
            "mean_ms": round(statistics.fmean(lat), 3) if lat else None,
            "frames_per_s": round(len(lat) / wall, 2) if wall > 0 else None,
            "rays_per_s": round(rays / wall, 1) if wall > 0 else None,
            "retries": sum(r.retries for r in reqs)}
