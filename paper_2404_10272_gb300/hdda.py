"""Thin ctypes binding of libhdda (``include/hdda.h``).

Argument marshalling only: every step of the sampler runs in the CUDA
library.  Tensors are torch CUDA tensors (device memory and streams come
from PyTorch); calls run on the current torch stream.  There is no CPU
fallback: if the library is not built, or a call fails, an exception says
so.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

OK = 0
ERR_INVALID_ARG, ERR_CUDA, ERR_CAPACITY, ERR_STEP_LIMIT, ERR_TIMEOUT, ERR_OOM, ERR_INTERNAL = range(1, 8)
GRID_DENSE, GRID_VDB = 0, 1
WALK_BRANCH, WALK_SKIP = 0, 1
SAMPLER_SEPARATE, SAMPLER_FUSED = 0, 1
(ARRAY_THRESHOLDS, ARRAY_DENSE_BITS, ARRAY_CHILD_MASK, ARRAY_TILE_MASK, ARRAY_LEAF_PREFIX,
 ARRAY_LEAVES, ARRAY_NODE_SUPER, ARRAY_LEAF_SUB, ARRAY_REGION_MAP) = range(9)

EXPORTED = [
    "hdda_version", "hdda_last_error", "hdda_pack_dense", "hdda_build_vdb", "hdda_grid_rebuild",
    "hdda_grid_stats_get", "hdda_grid_copy_array", "hdda_grid_free", "hdda_traverse_dense",
    "hdda_traverse_hdda", "hdda_composite", "hdda_profiler_enable", "hdda_profiler_read",
    "hdda_traverse_hdda_noalloc", "hdda_grid_set_refine", "hdda_batch_create",
    "hdda_batch_launch", "hdda_batch_results", "hdda_batch_free", "hdda_grid_set_walk",
    "hdda_render", "hdda_grid_update", "hdda_traverse_async", "hdda_set_region_checks",
    "hdda_region_checks", "hdda_traverse_composite", "hdda_set_sampler_form",
    "hdda_sampler_form",
]


class HddaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libhdda status {code}: {msg}")
        self.code = code


class AABB(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class Params(ctypes.Structure):
    _fields_ = [("near_t", ctypes.c_float), ("far_t", ctypes.c_float), ("step", ctypes.c_float),
                ("cone_angle", ctypes.c_float), ("max_step", ctypes.c_float),
                ("max_steps", ctypes.c_int32), ("image_width", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class Job(ctypes.Structure):
    _fields_ = [("rays_o", ctypes.c_void_p), ("rays_d", ctypes.c_void_p), ("n_rays", ctypes.c_int64),
                ("grid", ctypes.c_void_p), ("params", Params), ("offsets", ctypes.c_void_p),
                ("ray_idx", ctypes.c_void_p), ("t0", ctypes.c_void_p), ("t1", ctypes.c_void_p),
                ("capacity", ctypes.c_int64)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("walk_block", ctypes.c_int32), ("rays_per_fetch", ctypes.c_int32),
                ("emit_warps", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("walk_variant", ctypes.c_int32)]


class GridStats(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("levels", ctypes.c_int32), ("res", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("nodes", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_leaves", ctypes.c_int64), ("n_tiles", ctypes.c_int64), ("bytes", ctypes.c_int64),
                ("dense_bytes", ctypes.c_int64), ("map_bytes", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.library_path()


def load(path: str | None = None):
    """Loads libhdda.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libhdda is not built ({p} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    lib.hdda_version.restype = ctypes.c_char_p
    lib.hdda_last_error.restype = ctypes.c_char_p
    lib.hdda_pack_dense.argtypes = [vp, i32, i32, ctypes.POINTER(AABB), ctypes.POINTER(vp), vp]
    lib.hdda_build_vdb.argtypes = [vp, i32, i32, ctypes.POINTER(AABB), ctypes.POINTER(vp),
                                   ctypes.POINTER(sz), vp]
    lib.hdda_grid_rebuild.argtypes = [vp, vp, vp]
    lib.hdda_grid_update.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.hdda_grid_stats_get.argtypes = [vp, ctypes.POINTER(GridStats)]
    lib.hdda_grid_copy_array.argtypes = [vp, i32, vp, sz, ctypes.POINTER(sz)]
    lib.hdda_grid_set_refine.argtypes = [vp, i32]
    lib.hdda_grid_set_walk.argtypes = [vp, i32]
    lib.hdda_batch_create.argtypes = [ctypes.POINTER(Job), i32, ctypes.POINTER(BatchConfig),
                                      ctypes.POINTER(vp), vp]
    lib.hdda_batch_launch.argtypes = [vp, vp]
    lib.hdda_batch_results.argtypes = [vp, vp, vp, vp]
    lib.hdda_batch_free.argtypes = [vp]
    lib.hdda_batch_free.restype = None
    lib.hdda_grid_free.argtypes = [vp]
    lib.hdda_grid_free.restype = None
    trav = [vp, vp, i64, vp, ctypes.POINTER(Params), vp, vp, vp, vp, i64, ctypes.POINTER(i64), vp]
    lib.hdda_traverse_dense.argtypes = trav
    lib.hdda_traverse_hdda.argtypes = trav
    lib.hdda_traverse_hdda_noalloc.argtypes = trav
    lib.hdda_composite.argtypes = [vp, vp, i64, vp, vp, vp, vp, i32, vp, vp]
    lib.hdda_render.argtypes = [vp, vp, i64, vp, ctypes.POINTER(Params), vp, i32, vp, vp, vp]
    lib.hdda_traverse_async.argtypes = [vp, vp, i64, vp, ctypes.POINTER(Params), vp, vp, vp, vp,
                                        i64, vp, vp]
    lib.hdda_traverse_composite.argtypes = [vp, vp, i64, vp, ctypes.POINTER(Params), vp, vp, vp,
                                            vp, i64, vp, i32, vp, vp, vp]
    lib.hdda_profiler_enable.argtypes = [i32]
    lib.hdda_profiler_read.argtypes = [ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
    for name in EXPORTED:
        if name not in ("hdda_version", "hdda_last_error", "hdda_grid_free", "hdda_batch_free"):
            getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _check(code: int):
    if code != OK:
        raise HddaError(code, load().hdda_last_error().decode())


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _hold(stream, *tensors):
    """Tensors read by work queued on `stream` (not the current one) stay allocated until
    that work is done: the caching allocator is told the stream uses them."""
    if stream is None:
        return
    for t in tensors:
        if isinstance(t, torch.Tensor) and t.is_cuda:
            t.record_stream(stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _cuda(t, dtype, shape=None):
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t))
    if t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
        t = t.to(device="cuda", dtype=dtype).contiguous()
    if shape is not None:
        t = t.reshape(shape)
    return t


def _aabbs(aabbs, levels):
    a = np.asarray(aabbs, np.float32).reshape(levels, 6)
    arr = (AABB * levels)()
    for l in range(levels):
        arr[l].lo[:] = [float(v) for v in a[l, :3]]
        arr[l].hi[:] = [float(v) for v in a[l, 3:]]
    return arr


def make_params(near, far, step, cone=0.0, max_step=1e10, max_steps=1 << 20,
                image_width=0) -> Params:
    return Params(near, far, step, cone, max_step, max_steps, image_width)


class Grid:
    """A library-owned device grid (dense bit array or VDB tree)."""

    def __init__(self, handle, kind, levels, res):
        self._h = handle
        self.kind, self.levels, self.res = kind, levels, res

    @property
    def handle(self):
        return self._h

    def stats(self) -> GridStats:
        st = GridStats()
        _check(load().hdda_grid_stats_get(self._h, ctypes.byref(st)))
        return st

    def array(self, which: int) -> np.ndarray:
        need = ctypes.c_size_t(0)
        _check(load().hdda_grid_copy_array(self._h, which, None, 0, ctypes.byref(need)))
        dt = {ARRAY_THRESHOLDS: np.float32, ARRAY_REGION_MAP: np.uint16}.get(which, np.uint32)
        out = np.zeros(need.value // np.dtype(dt).itemsize, dt)
        _check(load().hdda_grid_copy_array(self._h, which, out.ctypes.data_as(ctypes.c_void_p),
                                           out.nbytes, ctypes.byref(need)))
        return out

    def set_refine(self, on: bool):
        """VDB grids: walk the refined tree through its region map (True, default) or the
        plain tree (False)."""
        _check(load().hdda_grid_set_refine(self._h, 1 if on else 0))

    def set_walk(self, variant: int):
        """WALK_BRANCH (Algorithm 1, default) or WALK_SKIP (Algorithm 2) control flow."""
        _check(load().hdda_grid_set_walk(self._h, int(variant)))

    def rebuild(self, dense: torch.Tensor, stream=None):
        d = _cuda(dense, torch.uint8)
        _hold(stream, d)
        _check(load().hdda_grid_rebuild(self._h, _ptr(d), _stream(stream)))

    def update(self, dense: torch.Tensor, blocks: torch.Tensor | None = None,
               status: torch.Tensor | None = None, stream=None):
        """Incremental rebuild (hdda_grid_update): `blocks` is a CUDA int64 tensor of the
        8^3-block indices l*B^3 + (bx*B + by)*B + bz that may have changed (None: all)."""
        d = _cuda(dense, torch.uint8)
        bp, nb = None, 0
        if blocks is not None:
            b = _cuda(blocks, torch.int64)
            bp, nb = _ptr(b), int(b.numel())
        st = 0
        if status is not None:
            if not status.is_cuda or status.numel() < 1 or status.element_size() != 4:
                raise ValueError("status must be a CUDA tensor of 4-byte elements")
            st = status.data_ptr()
        _hold(stream, d, b if blocks is not None else None)
        _check(load().hdda_grid_update(self._h, _ptr(d), bp, nb, st, _stream(stream)))

    def free(self):
        if self._h:
            load().hdda_grid_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _dense_args(dense, aabbs):
    d = _cuda(dense, torch.uint8)
    if d.dim() == 3:
        d = d.unsqueeze(0)
    L, R = int(d.shape[0]), int(d.shape[1])
    if tuple(d.shape) != (L, R, R, R):
        raise ValueError(f"dense must be [L, R, R, R], got {tuple(d.shape)}")
    return d, L, R, _aabbs(aabbs, L)


def pack_dense(dense, aabbs, stream=None) -> Grid:
    d, L, R, boxes = _dense_args(dense, aabbs)
    h = ctypes.c_void_p()
    _hold(stream, d)
    _check(load().hdda_pack_dense(_ptr(d), L, R, boxes, ctypes.byref(h), _stream(stream)))
    return Grid(h, GRID_DENSE, L, R)


def build_vdb(dense, aabbs, stream=None) -> Grid:
    d, L, R, boxes = _dense_args(dense, aabbs)
    h = ctypes.c_void_p()
    _hold(stream, d)
    _check(load().hdda_build_vdb(_ptr(d), L, R, boxes, ctypes.byref(h), None, _stream(stream)))
    return Grid(h, GRID_VDB, L, R)


@dataclass
class Samples:
    offsets: torch.Tensor   # int64 [n+1]
    ray_idx: torch.Tensor   # int32 [capacity] (first `total` valid)
    t0: torch.Tensor        # float32 [capacity]
    t1: torch.Tensor        # float32 [capacity]
    total: int

    def trimmed(self):
        n = self.total
        return self.offsets, self.ray_idx[:n], self.t0[:n], self.t1[:n]


def alloc_samples(n_rays: int, capacity: int, device="cuda") -> Samples:
    return Samples(offsets=torch.empty(n_rays + 1, dtype=torch.int64, device=device),
                   ray_idx=torch.empty(capacity, dtype=torch.int32, device=device),
                   t0=torch.empty(capacity, dtype=torch.float32, device=device),
                   t1=torch.empty(capacity, dtype=torch.float32, device=device), total=0)


def _traverse(fn_name, rays_o, rays_d, grid: Grid, params: Params, out: Samples | None,
              count_only: bool, stream):
    ro = _cuda(rays_o, torch.float32, (-1, 3))
    rd = _cuda(rays_d, torch.float32, (-1, 3))
    n = int(ro.shape[0])
    fn = getattr(load(), fn_name)
    total = ctypes.c_int64(0)
    s = _stream(stream)
    if out is None:
        out = alloc_samples(n, 0, ro.device)
        _check(fn(_ptr(ro), _ptr(rd), n, grid.handle, ctypes.byref(params), _ptr(out.offsets),
                  None, None, None, 0, ctypes.byref(total), s))
        out.total = total.value
        if count_only:
            return out
        out = alloc_samples(n, max(1, total.value), ro.device)
    cap = 0 if count_only else int(out.t0.numel())
    code = fn(_ptr(ro), _ptr(rd), n, grid.handle, ctypes.byref(params), _ptr(out.offsets),
              _ptr(out.ray_idx), _ptr(out.t0), _ptr(out.t1), cap, ctypes.byref(total), s)
    out.total = total.value
    _check(code)
    return out


def traverse_dense(rays_o, rays_d, grid: Grid, params: Params, out: Samples | None = None,
                   count_only: bool = False, stream=None) -> Samples:
    """Dense-grid DDA sampler.  Without `out`, counts first and allocates
    exactly; with `out`, its capacity is used (HddaError ERR_CAPACITY if it
    is too small)."""
    return _traverse("hdda_traverse_dense", rays_o, rays_d, grid, params, out, count_only, stream)


def traverse_async(rays_o, rays_d, grid: Grid, params: Params, out: Samples,
                   status: torch.Tensor, stream=None) -> Samples:
    """Stream-ordered sampler (hdda_traverse_async): HDDA for a VDB grid, dense DDA for a
    dense grid.  Nothing is read back; `out.total` is left at -1 and the total is
    `out.offsets[-1]` on the device.  `status` is a CUDA tensor of one 4-byte element
    that receives status bits (2 = internal check failed, 4 = capacity below the total)."""
    ro = _cuda(rays_o, torch.float32, (-1, 3))
    rd = _cuda(rays_d, torch.float32, (-1, 3))
    if not status.is_cuda or status.numel() < 1 or status.element_size() != 4:
        raise ValueError("status must be a CUDA tensor of 4-byte elements")
    n = int(ro.shape[0])
    _hold(stream, ro, rd, out.offsets, out.ray_idx, out.t0, out.t1, status)
    _check(load().hdda_traverse_async(_ptr(ro), _ptr(rd), n, grid.handle, ctypes.byref(params),
                                      _ptr(out.offsets), _ptr(out.ray_idx), _ptr(out.t0),
                                      _ptr(out.t1), int(out.t0.numel()), status.data_ptr(),
                                      _stream(stream)))
    out.total = -1
    return out


def traverse_composite(rays_o, rays_d, grid: Grid, params: Params, out: Samples, field,
                       status: torch.Tensor, rgba: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    """Sampling and compositing fused (hdda_traverse_composite): writes the
    samples traverse_async writes into `out` and returns the frame render
    gives, from one stream-ordered call.  `status` as for traverse_async."""
    ro = _cuda(rays_o, torch.float32, (-1, 3))
    rd = _cuda(rays_d, torch.float32, (-1, 3))
    f = _cuda(field, torch.float32, (-1, 8))
    if not status.is_cuda or status.numel() < 1 or status.element_size() != 4:
        raise ValueError("status must be a CUDA tensor of 4-byte elements")
    n = int(ro.shape[0])
    if rgba is None:
        rgba = torch.empty((n, 4), dtype=torch.float32, device=ro.device)
    _hold(stream, ro, rd, f, out.offsets, out.ray_idx, out.t0, out.t1, status, rgba)
    _check(load().hdda_traverse_composite(
        _ptr(ro), _ptr(rd), n, grid.handle, ctypes.byref(params), _ptr(out.offsets),
        _ptr(out.ray_idx), _ptr(out.t0), _ptr(out.t1), int(out.t0.numel()), _ptr(f),
        int(f.shape[0]), _ptr(rgba), status.data_ptr(), _stream(stream)))
    out.total = -1
    return rgba


def traverse_hdda(rays_o, rays_d, grid: Grid, params: Params, out: Samples | None = None,
                  count_only: bool = False, stream=None) -> Samples:
    """Hierarchical-DDA sampler over a VDB grid (same contract)."""
    return _traverse("hdda_traverse_hdda", rays_o, rays_d, grid, params, out, count_only, stream)


def traverse_hdda_noalloc(rays_o, rays_d, grid: Grid, params: Params, out: Samples,
                          stream=None) -> Samples:
    """Hierarchical-DDA sampler that allocates no memory of its own (static
    device scratch inside the library).  `out` must be preallocated and
    large enough; calls whose GPU work overlaps must be serialised."""
    ro = _cuda(rays_o, torch.float32, (-1, 3))
    rd = _cuda(rays_d, torch.float32, (-1, 3))
    n = int(ro.shape[0])
    total = ctypes.c_int64(0)
    code = load().hdda_traverse_hdda_noalloc(
        _ptr(ro), _ptr(rd), n, grid.handle, ctypes.byref(params), _ptr(out.offsets),
        _ptr(out.ray_idx), _ptr(out.t0), _ptr(out.t1), int(out.t0.numel()), ctypes.byref(total),
        _stream(stream))
    out.total = total.value
    _check(code)
    return out


def composite(rays_o, rays_d, samples: Samples, field, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    ro = _cuda(rays_o, torch.float32, (-1, 3))
    rd = _cuda(rays_d, torch.float32, (-1, 3))
    f = _cuda(field, torch.float32, (-1, 8))
    n = int(ro.shape[0])
    if out is None:
        out = torch.empty((n, 4), dtype=torch.float32, device=ro.device)
    _hold(stream, ro, rd, f, samples.offsets, samples.t0, samples.t1, out)
    _check(load().hdda_composite(_ptr(ro), _ptr(rd), n, _ptr(samples.offsets), _ptr(samples.t0),
                                 _ptr(samples.t1), _ptr(f), int(f.shape[0]), _ptr(out),
                                 _stream(stream)))
    return out


def render(rays_o, rays_d, grid: Grid, params: Params, field, out: torch.Tensor | None = None,
           status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Render-only path (hdda_render): the frame that traverse + composite would
    give, without writing any sample.  A VDB grid is walked by HDDA, a dense
    grid by dense DDA.  With `status` (a CUDA int32/uint32 tensor of one
    element) the call does not synchronise and device status bits are ORed
    into it; without it the call checks them before returning."""
    ro = _cuda(rays_o, torch.float32, (-1, 3))
    rd = _cuda(rays_d, torch.float32, (-1, 3))
    f = _cuda(field, torch.float32, (-1, 8))
    n = int(ro.shape[0])
    if out is None:
        out = torch.empty((n, 4), dtype=torch.float32, device=ro.device)
    st = 0
    if status is not None:
        if not status.is_cuda or status.numel() < 1 or status.element_size() != 4:
            raise ValueError("status must be a CUDA tensor of 4-byte elements")
        st = status.data_ptr()
    _hold(stream, ro, rd, f, out, status)
    _check(load().hdda_render(_ptr(ro), _ptr(rd), n, grid.handle, ctypes.byref(params), _ptr(f),
                              int(f.shape[0]), _ptr(out), st, _stream(stream)))
    return out


PROFILE_TIMERS = 1
PROFILE_COUNTERS = 2


def profiler_enable(on: bool = True, counters: bool = False):
    """Kernel timers on or off; `counters` also turns on the work counters
    (extra device work: time with the timers alone)."""
    flags = (PROFILE_TIMERS if on else 0) | (PROFILE_COUNTERS if counters else 0)
    _check(load().hdda_profiler_enable(flags))


def set_region_checks(on: bool = True):
    """Device-side region checks on or off (process-wide, off by default):
    while on, a walk that finds a region not holding its point raises
    HDDA_ERR_INTERNAL (or bit 1 of a device status word)."""
    _check(load().hdda_set_region_checks(1 if on else 0))


def region_checks() -> bool:
    """The current region-check setting."""
    return bool(load().hdda_region_checks())


def set_sampler_form(form: int):
    """Form of the two-pass samplers (process-wide): SAMPLER_SEPARATE
    (default: the walk and the emit as two kernels) or SAMPLER_FUSED (both
    passes in one persistent kernel).  Both give the same samples."""
    _check(load().hdda_set_sampler_form(int(form)))


def sampler_form() -> int:
    """The current sampler form."""
    return int(load().hdda_sampler_form())


def profiler_read() -> dict:
    """{kernel name: (launches, total ms)} since the last read (synchronises)."""
    cap = 64
    arr = (KernelTime * cap)()
    n = ctypes.c_int(0)
    _check(load().hdda_profiler_read(arr, cap, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(n.value, cap))}


DEFAULT_BATCH_CONFIG = (256, 64, 4)


class Batch:
    """A batch plan over many traversal jobs (see hdda_batch_create).

    jobs: list of dicts with rays_o, rays_d (CUDA float32 [n, 3]), grid (Grid),
    params (Params) and out (Samples: offsets [n+1] and sample buffers whose
    length is the job's capacity).  The tensors and grids are kept alive
    by the batch.  config: (walk_block, rays_per_fetch, emit_warps[,
    walk_variant]) with walk_variant WALK_BRANCH (default) or WALK_SKIP.
    """

    def __init__(self, jobs, config=DEFAULT_BATCH_CONFIG, use_graph=True, stream=None):
        self._keep = []
        arr = (Job * len(jobs))()
        for i, jb in enumerate(jobs):
            ro = _cuda(jb["rays_o"], torch.float32, (-1, 3))
            rd = _cuda(jb["rays_d"], torch.float32, (-1, 3))
            out = jb["out"]
            self._keep += [ro, rd, out, jb["grid"]]
            arr[i] = Job(_ptr(ro), _ptr(rd), int(ro.shape[0]), jb["grid"].handle, jb["params"],
                         _ptr(out.offsets), _ptr(out.ray_idx), _ptr(out.t0), _ptr(out.t1),
                         int(out.t0.numel()))
        self.n_jobs = len(jobs)
        self.jobs = jobs
        wb, rpf, ew = config[:3]
        wv = config[3] if len(config) > 3 else WALK_BRANCH
        cfg = BatchConfig(wb, rpf, ew, 1 if use_graph else 0, wv)
        self.config = (wb, rpf, ew, wv)
        h = ctypes.c_void_p()
        _check(load().hdda_batch_create(arr, self.n_jobs, ctypes.byref(cfg), ctypes.byref(h),
                                        _stream(stream)))
        self._h = h

    def launch(self, stream=None):
        _check(load().hdda_batch_launch(self._h, _stream(stream)))

    def results(self, stream=None, check=True):
        """(totals, status) per job after the last launch (synchronises)."""
        totals = (ctypes.c_int64 * self.n_jobs)()
        status = (ctypes.c_uint32 * self.n_jobs)()
        code = load().hdda_batch_results(self._h, totals, status, _stream(stream))
        tot, st = list(totals), list(status)
        for jb, t in zip(self.jobs, tot):
            jb["out"].total = t
        if check:
            _check(code)
        return tot, st

    def free(self):
        if self._h:
            load().hdda_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
