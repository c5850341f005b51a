"""Shared helpers for the GPU parity tests (not collected by pytest)."""
import numpy as np

import oracle


def to_np(t):
    return t.detach().cpu().numpy()


def gpu_samples(hdda, kind, o, d, grid, params, out=None):
    fn = hdda.traverse_hdda if kind == "hdda" else hdda.traverse_dense
    s = fn(o, d, grid, params, out=out)
    off, idx, t0, t1 = s.trimmed()
    return to_np(off), to_np(idx), to_np(t0), to_np(t1)


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
