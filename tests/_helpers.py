"""Shared helpers for the GPU parity tests (not collected by pytest)."""
import contextlib

import numpy as np

import oracle
from paper_2404_10272_gb300 import scenes


def to_np(t):
    return t.detach().cpu().numpy()


def gpu_samples(hdda, kind, o, d, grid, params, out=None):
    fn = hdda.traverse_hdda if kind == "hdda" else hdda.traverse_dense
    s = fn(o, d, grid, params, out=out)
    off, idx, t0, t1 = s.trimmed()
    return to_np(off), to_np(idx), to_np(t0), to_np(t1)


@contextlib.contextmanager
def sampler_form(hdda, form):
    """Runs the block with the two-pass samplers in `form` (SAMPLER_SEPARATE or
    SAMPLER_FUSED), then restores the previous form."""
    before = hdda.sampler_form()
    hdda.set_sampler_form(form)
    try:
        yield
    finally:
        hdda.set_sampler_form(before)


def oracle_samples(o, d, occ, aabbs, p):
    return oracle.sample(o, d, occ, aabbs, p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)


def assert_same(a, b, what=""):
    """Bit-exact equality of two (offsets, ray_idx, t0, t1) sample sets."""
    off_a, idx_a, t0_a, t1_a = a
    off_b, idx_b, t0_b, t1_b = b
    assert np.array_equal(off_a, off_b), f"{what}: offsets differ"
    assert np.array_equal(idx_a, idx_b), f"{what}: ray_idx differ"
    assert np.array_equal(np.ascontiguousarray(t0_a).view(np.uint32),
                          np.ascontiguousarray(t0_b).view(np.uint32)), f"{what}: t0 differ"
    assert np.array_equal(np.ascontiguousarray(t1_a).view(np.uint32),
                          np.ascontiguousarray(t1_b).view(np.uint32)), f"{what}: t1 differ"


def subset_rays(o, d, stride, offset=0):
    sel = np.arange(offset, o.shape[0], stride)
    return np.ascontiguousarray(o[sel]), np.ascontiguousarray(d[sel]), sel


def slab_scene(R, period, n_rays, seed):
    """Occupied x-slabs every `period` voxels: rays along +x cross R / period
    separate runs, so they need several rounds of kMaxRuns = 16 runs."""
    rng = np.random.default_rng(seed)
    occ = np.zeros((1, R, R, R), np.uint8)
    occ[0, ::period] = 1
    aabbs = np.array([[0, 0, 0, 1, 1, 1]], np.float32)
    o = np.empty((n_rays, 3), np.float32)
    o[:, 0] = -0.25
    o[:, 1:] = rng.uniform(0.05, 0.95, (n_rays, 2))
    d = np.empty((n_rays, 3), np.float64)
    d[:, 0] = 1.0
    d[:, 1:] = rng.uniform(-0.15, 0.15, (n_rays, 2))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = d.astype(np.float32)
    # faint blobs over the box: transmittance stays well above 0 to the far side
    field = np.zeros((8, 8), np.float32)
    field[:, :3] = rng.uniform(0.1, 0.9, (8, 3))
    field[:, 3] = rng.uniform(0.2, 0.4, 8)
    field[:, 4] = rng.uniform(0.5, 2.0, 8)
    field[:, 5:] = rng.uniform(0, 1, (8, 3))
    p = scenes.SamplerParams(near=0.0, far=1.6, step=1.0 / 512, cone=0.0, max_step=1e10,
                             max_steps=1 << 20)
    return occ, aabbs, o, d, field, p
