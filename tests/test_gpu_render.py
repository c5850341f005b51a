"""Render-only path (hdda_render): the frame of sampling + compositing without
stored samples.  Pixels are checked against the binary64 oracle compositor
over the oracle's own samples (|error| <= 1e-5 per channel), and the
walk-method invariance is checked bit for bit: dense DDA, HDDA with and
without refinement and the Algorithm 2 control flow keep the same intervals
and number them the same way, so their frames are identical."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_10272_gb300 import scenes
from _helpers import oracle_samples, slab_scene as _slab_scene, subset_rays, to_np

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


def _oracle_frame(sc, o, d):
    off, _, t0, t1 = oracle_samples(o, d, sc.occ, sc.aabbs, sc.params)
    return oracle.composite(o, d, off, t0, t1, sc.field), off


def _check_scene(H, sc, o, d):
    ref, off = _oracle_frame(sc, o, d)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(sc.field).cuda()
    prm = _params(H, sc.params)
    occ = torch.from_numpy(sc.occ).cuda()
    gv = H.build_vdb(occ, sc.aabbs)
    rgba = to_np(H.render(ot, dt, gv, prm, f))
    err = np.abs(rgba.astype(np.float64) - ref)
    assert err.max() <= TOL, err.max()
    # every walk keeps the same runs: identical frames
    gd = H.pack_dense(occ, sc.aabbs)
    assert np.array_equal(to_np(H.render(ot, dt, gd, prm, f)).view(np.uint32), rgba.view(np.uint32))
    gv.set_refine(False)
    assert np.array_equal(to_np(H.render(ot, dt, gv, prm, f)).view(np.uint32), rgba.view(np.uint32))
    gv.set_refine(True)
    gv.set_walk(H.WALK_SKIP)
    assert np.array_equal(to_np(H.render(ot, dt, gv, prm, f)).view(np.uint32), rgba.view(np.uint32))
    # beside traverse + composite (different chunking, same sums up to rounding)
    gv.set_walk(H.WALK_BRANCH)
    s = H.traverse_hdda(ot, dt, gv, prm)
    two = to_np(H.composite(ot, dt, s, f)).astype(np.float64)
    assert np.abs(two - rgba).max() <= 2 * TOL
    return ref, off


def test_tiny_frame(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    ref, _ = _check_scene(H, sc, o, d)
    assert ref[:, 3].max() > 0.5


def test_object_frame_subset(H):
    sc = scenes.object_scene()
    o, d = scenes.object_cameras(n=1)[0].rays()
    o, d, _ = subset_rays(o, d, 53, 11)
    _check_scene(H, sc, o, d)


def test_unbounded_frame_subset(H):
    sc = scenes.unbounded_scene()
    o, d = scenes.unbounded_camera().rays()
    o, d, _ = subset_rays(o, d, 97, 5)
    _check_scene(H, sc, o, d)


@pytest.mark.parametrize("R,period", [(64, 2), (128, 2), (128, 5)])
def test_rays_with_many_runs(H, R, period):
    occ, aabbs, o, d, field, p = _slab_scene(R, period, 700, 7000 + R + period)
    off, _, t0, t1 = oracle.sample(o, d, occ, aabbs, p.near, p.far, p.step, p.cone, p.max_step,
                                   p.max_steps)
    ref = oracle.composite(o, d, off, t0, t1, field)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(field).cuda()
    prm = _params(H, p)
    g = H.build_vdb(torch.from_numpy(occ).cuda(), aabbs)
    rgba = to_np(H.render(ot, dt, g, prm, f))
    assert np.abs(rgba.astype(np.float64) - ref).max() <= TOL
    # most rays need more than one round, and light still gets through at the far end
    runs = np.array([1 + int(np.sum(t0[off[r] + 1:off[r + 1]] != t1[off[r]:off[r + 1] - 1]))
                     if off[r + 1] > off[r] else 0 for r in range(o.shape[0])])
    assert (runs > 16).mean() > 0.5 and ref[:, 3].max() < 0.95
    gd = H.pack_dense(torch.from_numpy(occ).cuda(), aabbs)
    assert np.array_equal(to_np(H.render(ot, dt, gd, prm, f)).view(np.uint32), rgba.view(np.uint32))


def test_async_status_mode(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(sc.field).cuda()
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    prm = _params(H, sc.params)
    sync = to_np(H.render(ot, dt, g, prm, f))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        out = H.render(ot, dt, g, prm, f, status=status, stream=stream)
    stream.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(to_np(out).view(np.uint32), sync.view(np.uint32))


def test_edges(H):
    sc = scenes.tiny_scene()
    f = torch.from_numpy(sc.field).cuda()
    prm = _params(H, sc.params)
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    assert H.render(empty, empty, g, prm, f).shape == (0, 4)
    # no occupied voxel: transparent black
    ge = H.build_vdb(torch.zeros_like(torch.from_numpy(sc.occ)).cuda(), sc.aabbs)
    o, d = scenes.tiny_camera().rays()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    assert float(H.render(ot, dt, ge, prm, f).abs().max()) == 0.0
    # non-finite rays and zero directions have no samples; a ragged count of rays
    o2 = np.array(o[:37])
    d2 = np.array(d[:37])
    o2[3] = np.nan
    d2[4] = np.inf
    d2[5] = 0.0
    rgba = to_np(H.render(torch.from_numpy(o2).cuda(), torch.from_numpy(d2).cuda(), g, prm, f))
    ref, _ = _oracle_frame(sc, o2, d2)
    assert np.all(rgba[3:6] == 0.0)
    assert np.abs(rgba.astype(np.float64) - ref).max() <= TOL
    # no blobs: nothing is emitted
    z = torch.zeros((0, 8), dtype=torch.float32, device="cuda")
    assert float(H.render(ot, dt, g, prm, z).abs().max()) == 0.0
    with pytest.raises(H.HddaError):
        H.render(ot, dt, g, prm, torch.zeros((257, 8), dtype=torch.float32, device="cuda"))


def test_counters_leave_pixels_unchanged(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(sc.field).cuda()
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    prm = _params(H, sc.params)
    plain = to_np(H.render(ot, dt, g, prm, f))
    s = H.traverse_hdda(ot, dt, g, prm)
    comp = to_np(H.composite(ot, dt, s, f))
    H.profiler_read()
    H.profiler_enable(True, counters=True)
    try:
        counted = to_np(H.render(ot, dt, g, prm, f))
        counted_c = to_np(H.composite(ot, dt, s, f))
    finally:
        H.profiler_enable(False)
    got = H.profiler_read()
    assert np.array_equal(counted.view(np.uint32), plain.view(np.uint32))
    assert np.array_equal(counted_c.view(np.uint32), comp.view(np.uint32))
    # culling keeps at most every blob for every sample
    n_samples = s.total
    for name in ("render_blob_evals", "composite_blob_evals"):
        ev = got[name][0]
        assert 0 < ev <= n_samples * sc.field.shape[0], (name, ev)
    assert got["hdda_render"][0] == 1 and got["composite"][0] == 1
