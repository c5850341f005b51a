"""Stream-ordered traversal (hdda_traverse_async): the same offsets and samples as
the synchronous samplers, bit for bit, on dense and VDB grids; a capacity below the
total raises the status bit, writes nothing past capacity and clamps the offsets
(the synchronous samplers clamp them too), so the compositor queued behind it stays
in bounds."""
import numpy as np
import pytest
import torch

from paper_2404_10272_gb300 import scenes
from _helpers import assert_same, sampler_form, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


@pytest.fixture(scope="module")
def frame(H):
    sc = scenes.object_scene()
    o, d = scenes.object_cameras(n=1)[0].rays()
    o, d = o[::7].copy(), d[::7].copy()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    occ = torch.from_numpy(sc.occ).cuda()
    p = sc.params
    prm = H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    return sc, ot, dt, occ, prm


def _trim(s, total):
    return (to_np(s.offsets), to_np(s.ray_idx[:total]), to_np(s.t0[:total]), to_np(s.t1[:total]))


@pytest.mark.parametrize("kind", ["vdb", "dense"])
def test_async_equals_sync(H, frame, kind):
    sc, ot, dt, occ, prm = frame
    g = H.build_vdb(occ, sc.aabbs) if kind == "vdb" else H.pack_dense(occ, sc.aabbs)
    sync = (H.traverse_hdda if kind == "vdb" else H.traverse_dense)(ot, dt, g, prm)
    ref = tuple(to_np(x) for x in sync.trimmed())
    out = H.alloc_samples(ot.shape[0], sync.total + 3)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        H.traverse_async(ot, dt, g, prm, out, st, stream=side)
        rgba = H.composite(ot, dt, out, torch.from_numpy(sc.field).cuda(), stream=side)
    side.synchronize()
    assert int(st.item()) == 0
    total = int(out.offsets[-1].item())
    assert total == sync.total
    assert_same(_trim(out, total), ref, f"async {kind}")
    two = H.composite(ot, dt, sync, torch.from_numpy(sc.field).cuda())
    assert torch.equal(rgba, two)
    # count only: offsets without samples, nothing clamped
    cnt = H.alloc_samples(ot.shape[0], 0)
    st.zero_()
    H.traverse_async(ot, dt, g, prm, cnt, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    np.testing.assert_array_equal(to_np(cnt.offsets), ref[0])


@pytest.mark.parametrize("form", ["separate", "fused"])
def test_capacity_overflow_clamps_offsets(H, frame, form):
    with sampler_form(H, H.SAMPLER_FUSED if form == "fused" else H.SAMPLER_SEPARATE):
        _capacity_overflow(H, frame)


def _capacity_overflow(H, frame):
    sc, ot, dt, occ, prm = frame
    g = H.build_vdb(occ, sc.aabbs)
    full = H.traverse_hdda(ot, dt, g, prm)
    ref = tuple(to_np(x) for x in full.trimmed())
    for cap in (full.total // 2, full.total - 1, 1):
        big = H.alloc_samples(ot.shape[0], full.total)
        big.t0.fill_(-1.0)
        view = H.Samples(big.offsets, big.ray_idx[:cap], big.t0[:cap], big.t1[:cap], 0)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        H.traverse_async(ot, dt, g, prm, view, st)
        rgba = H.composite(ot, dt, view, torch.from_numpy(sc.field).cuda())
        torch.cuda.synchronize()
        assert int(st.item()) == 4
        off = to_np(big.offsets)
        np.testing.assert_array_equal(off, np.minimum(ref[0], cap))
        np.testing.assert_array_equal(to_np(big.t0[:cap]).view(np.uint32), ref[2][:cap].view(np.uint32))
        assert bool((big.t0[cap:] == -1.0).all())
        assert bool(torch.isfinite(rgba).all())
    # the synchronous sampler reports the error and clamps the same way
    cap = full.total // 3
    big = H.alloc_samples(ot.shape[0], full.total)
    view = H.Samples(big.offsets, big.ray_idx[:cap], big.t0[:cap], big.t1[:cap], 0)
    with pytest.raises(H.HddaError) as ex:
        H.traverse_hdda(ot, dt, g, prm, out=view)
    assert ex.value.code == H.ERR_CAPACITY and view.total == full.total
    np.testing.assert_array_equal(to_np(big.offsets), np.minimum(ref[0], cap))


def test_async_argument_errors(H, frame):
    sc, ot, dt, occ, prm = frame
    g = H.build_vdb(occ, sc.aabbs)
    out = H.alloc_samples(ot.shape[0], 16)
    with pytest.raises(ValueError):
        H.traverse_async(ot, dt, g, prm, out, torch.zeros(1, dtype=torch.int64, device="cuda"))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    e = H.alloc_samples(0, 1)
    H.traverse_async(empty, empty, g, prm, e, st)
    torch.cuda.synchronize()
    assert int(e.offsets[0].item()) == 0 and int(st.item()) == 0
