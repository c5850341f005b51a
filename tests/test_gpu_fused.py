"""Sampling and compositing fused (hdda_traverse_composite): its offsets and
samples equal the stream-ordered sampler's bit for bit, its frame equals the
render-only path's bit for bit (and the binary64 oracle's within 1e-5), on
full frames, on rays that need several rounds of runs, on dense grids, with a
buffer too small and with none."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_10272_gb300 import scenes
from _helpers import slab_scene as _slab_scene, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


def _params(H, p):
    return H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)


def _both(H, ot, dt, g, prm, f, cap):
    """(fused samples, fused frame, fused status), (async samples, render frame)."""
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    fused = H.alloc_samples(ot.shape[0], cap)
    rgba = H.traverse_composite(ot, dt, g, prm, fused, f, st)
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    ref = H.alloc_samples(ot.shape[0], cap)
    H.traverse_async(ot, dt, g, prm, ref, st2)
    frame = H.render(ot, dt, g, prm, f)
    torch.cuda.synchronize()
    assert int(st.item()) == int(st2.item())
    return fused, rgba, int(st.item()), ref, frame


def _assert_samples_equal(a, b, total):
    np.testing.assert_array_equal(to_np(a.offsets), to_np(b.offsets))
    np.testing.assert_array_equal(to_np(a.ray_idx[:total]), to_np(b.ray_idx[:total]))
    np.testing.assert_array_equal(to_np(a.t0[:total]).view(np.uint32),
                                  to_np(b.t0[:total]).view(np.uint32))
    np.testing.assert_array_equal(to_np(a.t1[:total]).view(np.uint32),
                                  to_np(b.t1[:total]).view(np.uint32))


@pytest.mark.parametrize("which", ["object", "unbounded", "tiny"])
def test_full_frames(H, which):
    if which == "object":
        sc = scenes.object_scene()
        o, d = scenes.object_cameras(n=1)[0].rays()
        stride = 211
    elif which == "unbounded":
        sc = scenes.unbounded_scene()
        o, d = scenes.unbounded_camera().rays()
        stride = 1009
    else:
        sc = scenes.tiny_scene()
        o, d = scenes.tiny_camera().rays()
        stride = 7
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(sc.field).cuda()
    prm = _params(H, sc.params)
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    total = H.traverse_hdda(ot, dt, g, prm, count_only=True).total
    fused, rgba, st, ref, frame = _both(H, ot, dt, g, prm, f, total)
    assert st == 0
    assert int(fused.offsets[-1].item()) == total
    _assert_samples_equal(fused, ref, total)
    assert torch.equal(rgba, frame)
    off, t0, t1 = to_np(fused.offsets), to_np(fused.t0[:total]), to_np(fused.t1[:total])
    sel = np.arange(stride // 3, o.shape[0], stride)
    sub_off = np.concatenate([[0], np.cumsum(off[sel + 1] - off[sel])])
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in sel])
    want = oracle.composite(o[sel], d[sel], sub_off, t0[idx], t1[idx], sc.field)
    assert np.abs(to_np(rgba)[sel].astype(np.float64) - want).max() <= TOL


@pytest.mark.parametrize("R,period,kind", [(64, 2, "vdb"), (128, 5, "vdb"), (128, 2, "dense")])
def test_rays_in_several_rounds(H, R, period, kind):
    occ, aabbs, o, d, field, p = _slab_scene(R, period, 701, 9000 + R + period)
    ref_off, ref_idx, ref_t0, ref_t1 = oracle.sample(o, d, occ, aabbs, p.near, p.far, p.step,
                                                     p.cone, p.max_step, p.max_steps)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(field).cuda()
    prm = _params(H, p)
    dense = torch.from_numpy(occ).cuda()
    g = H.build_vdb(dense, aabbs) if kind == "vdb" else H.pack_dense(dense, aabbs)
    total = int(ref_off[-1])
    fused, rgba, st, ref, frame = _both(H, ot, dt, g, prm, f, total + 5)
    assert st == 0
    _assert_samples_equal(fused, ref, total)
    np.testing.assert_array_equal(to_np(fused.offsets), ref_off)
    np.testing.assert_array_equal(to_np(fused.ray_idx[:total]), ref_idx)
    np.testing.assert_array_equal(to_np(fused.t0[:total]).view(np.uint32), ref_t0.view(np.uint32))
    assert torch.equal(rgba, frame)
    want = oracle.composite(o, d, ref_off, ref_t0, ref_t1, field)
    assert np.abs(to_np(rgba).astype(np.float64) - want).max() <= TOL


def test_capacity_below_total_and_count_only(H):
    sc = scenes.object_scene()
    o, d = scenes.object_cameras(n=1)[0].rays()
    o, d = o[::5].copy(), d[::5].copy()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(sc.field).cuda()
    prm = _params(H, sc.params)
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    full = H.traverse_hdda(ot, dt, g, prm)
    frame = H.render(ot, dt, g, prm, f)
    for cap in (full.total // 2, full.total - 1, 0):
        big = H.alloc_samples(ot.shape[0], max(full.total, 1))
        big.t0.fill_(-1.0)
        view = H.Samples(big.offsets, big.ray_idx[:cap], big.t0[:cap], big.t1[:cap], 0)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        rgba = H.traverse_composite(ot, dt, g, prm, view, f, st)
        torch.cuda.synchronize()
        # capacity 0 counts only (offsets unclamped, no status), as the samplers do
        assert int(st.item()) == (4 if cap > 0 else 0)
        want_off = np.minimum(to_np(full.offsets), cap) if cap > 0 else to_np(full.offsets)
        np.testing.assert_array_equal(to_np(big.offsets), want_off)
        if cap > 0:
            np.testing.assert_array_equal(to_np(big.t0[:cap]).view(np.uint32),
                                          to_np(full.t0[:cap]).view(np.uint32))
        assert bool((big.t0[cap:] == -1.0).all())
        assert torch.equal(rgba, frame)   # the frame does not depend on the buffer


def test_arguments(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(sc.field).cuda()
    prm = _params(H, sc.params)
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    out = H.alloc_samples(ot.shape[0], 16)
    with pytest.raises(ValueError):
        H.traverse_composite(ot, dt, g, prm, out, f, torch.zeros(1, dtype=torch.int64,
                                                                 device="cuda"))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    e = H.alloc_samples(0, 1)
    rgba = H.traverse_composite(empty, empty, g, prm, e, f, st)
    torch.cuda.synchronize()
    assert rgba.shape == (0, 4) and int(e.offsets[0].item()) == 0 and int(st.item()) == 0
