"""GPU compositing against the binary64 oracle: |error| <= 1e-5 per channel
(binary32 field evaluation and accumulation)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2404_10272_gb300 import scenes
from _helpers import to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


def _render(H, sc, o, d):
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    p = sc.params
    prm = H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    s = H.traverse_hdda(ot, dt, g, prm)
    rgba = H.composite(ot, dt, s, torch.from_numpy(sc.field).cuda())
    off, idx, t0, t1 = (to_np(x) for x in s.trimmed())
    return to_np(rgba), off, t0, t1


def test_tiny_frame_matches_fp64_oracle(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    rgba, off, t0, t1 = _render(H, sc, o, d)
    ref = oracle.composite(o, d, off, t0, t1, sc.field)
    err = np.abs(rgba.astype(np.float64) - ref)
    assert err.max() <= TOL, err.max()
    assert ref[:, 3].max() > 0.5   # the frame is not trivially empty


def test_object_frame_subset_matches_fp64_oracle(H):
    sc = scenes.object_scene()
    o, d = scenes.object_cameras(n=1)[0].rays()
    rgba, off, t0, t1 = _render(H, sc, o, d)
    sel = np.arange(11, o.shape[0], 53)
    sub_off = np.concatenate([[0], np.cumsum(off[sel + 1] - off[sel])])
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in sel])
    ref = oracle.composite(o[sel], d[sel], sub_off, t0[idx], t1[idx], sc.field)
    err = np.abs(rgba[sel].astype(np.float64) - ref)
    assert err.max() <= TOL, err.max()


def test_composite_closed_forms(H):
    # constant field: one blob with a huge radius
    field = torch.tensor([[0, 0, 0, 1e6, 3.0, 0.2, 0.5, 0.9]], dtype=torch.float32, device="cuda")
    o = torch.zeros((3, 3), dtype=torch.float32, device="cuda")
    d = torch.tensor([[1, 0, 0]] * 3, dtype=torch.float32, device="cuda")
    s = H.alloc_samples(3, 5)
    s.offsets.copy_(torch.tensor([0, 0, 1, 5]))
    s.t0.copy_(torch.tensor([0.0, 0.25, 0.5, 1.0, 2.0]))
    s.t1.copy_(torch.tensor([0.25, 0.5, 0.75, 1.5, 2.125]))
    s.total = 5
    rgba = to_np(H.composite(o, d, s, field)).astype(np.float64)
    c = np.array([0.2, 0.5, 0.9], np.float32).astype(np.float64)
    np.testing.assert_array_equal(rgba[0], 0.0)
    a1 = 1 - math.exp(-0.75)
    np.testing.assert_allclose(rgba[1], [*(a1 * c), a1], atol=TOL)
    a = 1 - math.exp(-3.0 * 1.125)
    np.testing.assert_allclose(rgba[2], [*(a * c), a], atol=TOL)


def test_composite_no_blobs(H):
    o = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    d = torch.ones((2, 3), dtype=torch.float32, device="cuda")
    s = H.alloc_samples(2, 2)
    s.offsets.copy_(torch.tensor([0, 2, 2]))
    s.t0.copy_(torch.tensor([0.0, 1.0]))
    s.t1.copy_(torch.tensor([1.0, 2.0]))
    rgba = H.composite(o, d, s, torch.zeros((0, 8), dtype=torch.float32, device="cuda"))
    assert float(rgba.abs().max()) == 0.0


@pytest.mark.parametrize("which", ["object", "unbounded"])
def test_benchmark_step_full_size(H, which):
    """The step the benchmark times, at full size: grid rebuild, stream-ordered
    sampling into a preallocated buffer, compositing.  Its samples equal the
    synchronous sampler's bit for bit, and sampled pixels the binary64
    oracle's within 1e-5."""
    if which == "object":
        sc = scenes.object_scene()
        o, d = scenes.object_cameras(n=1)[0].rays()
        stride = 211
    else:
        sc = scenes.unbounded_scene()
        o, d = scenes.unbounded_camera().rays()
        stride = 1009
    p = sc.params
    prm = H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    dense = torch.from_numpy(sc.occ).cuda()
    field = torch.from_numpy(sc.field).cuda()
    g = H.build_vdb(dense, sc.aabbs)
    sync = H.traverse_hdda(ot, dt, g, prm)
    ref = tuple(to_np(x) for x in sync.trimmed())
    bufs = H.alloc_samples(ot.shape[0], sync.total)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    g.rebuild(dense)
    H.traverse_async(ot, dt, g, prm, bufs, st)
    rgba = H.composite(ot, dt, bufs, field)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    off = to_np(bufs.offsets)
    total = int(off[-1])
    assert total == sync.total
    t0 = to_np(bufs.t0[:total])
    t1 = to_np(bufs.t1[:total])
    np.testing.assert_array_equal(off, ref[0])
    np.testing.assert_array_equal(to_np(bufs.ray_idx[:total]), ref[1])
    np.testing.assert_array_equal(t0.view(np.uint32), ref[2].view(np.uint32))
    np.testing.assert_array_equal(t1.view(np.uint32), ref[3].view(np.uint32))
    sel = np.arange(stride // 3, o.shape[0], stride)
    sub_off = np.concatenate([[0], np.cumsum(off[sel + 1] - off[sel])])
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in sel])
    want = oracle.composite(o[sel], d[sel], sub_off, t0[idx], t1[idx], sc.field)
    err = np.abs(to_np(rgba)[sel].astype(np.float64) - want)
    assert err.max() <= TOL, err.max()
    assert want[:, 3].max() > 0.5


def _random_samples(rng, n_rays, counts):
    """Rays of random origin and (not unit) direction, one of them with a zero direction,
    and per ray `counts[r]` intervals in random order: non-negative lengths, some of length
    0, scattered over t in [0, 4)."""
    o = rng.uniform(-1.5, 1.5, (n_rays, 3)).astype(np.float32)
    d = rng.normal(size=(n_rays, 3)).astype(np.float32) * rng.uniform(0.5, 2.0, (n_rays, 1)).astype(np.float32)
    d[n_rays // 2] = 0.0
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S = int(off[-1])
    t0 = rng.uniform(0.0, 4.0, S).astype(np.float32)
    dt = rng.uniform(0.0, 0.02, S).astype(np.float32)
    dt[rng.random(S) < 0.05] = 0.0
    t1 = (t0 + dt).astype(np.float32)
    return o, d, off, t0, t1


@pytest.mark.parametrize("G", [1, 37, 64, 256])
def test_culling_paths_on_unordered_samples(H, G):
    # The compositor's culling takes different paths: chunks of one or two rays test blobs
    # against the rays' segments, chunks of three rays or more against their bounding box;
    # tasks longer than two chunks first narrow the field to the blobs near their rays'
    # lines.  Rays here hold 0, 1, a few or hundreds of samples, in random order along the
    # ray (the ABI does not ask for ascending t), so every path runs; pixels must stay within
    # 1e-5 of the binary64 oracle, which sums every blob.
    rng = np.random.default_rng(500 + G)
    counts = rng.choice([0, 1, 3, 17, 70, 300], size=203, p=[0.15, 0.15, 0.2, 0.2, 0.2, 0.1])
    o, d, off, t0, t1 = _random_samples(rng, counts.size, counts)
    field = np.zeros((G, 8), np.float32)
    field[:, :3] = rng.uniform(-2.0, 2.0, (G, 3))
    field[:, 3] = rng.uniform(0.03, 0.4, G)
    field[:, 4] = rng.uniform(0.5, 30.0, G)
    field[:, 5:] = rng.uniform(0.0, 1.0, (G, 3))
    s = H.alloc_samples(o.shape[0], max(1, int(off[-1])))
    s.offsets.copy_(torch.from_numpy(off))
    s.t0[:off[-1]].copy_(torch.from_numpy(t0))
    s.t1[:off[-1]].copy_(torch.from_numpy(t1))
    s.total = int(off[-1])
    rgba = to_np(H.composite(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), s,
                             torch.from_numpy(field).cuda())).astype(np.float64)
    ref = oracle.composite(o, d, off, t0, t1, field)
    assert np.abs(rgba - ref).max() <= TOL, np.abs(rgba - ref).max()
    assert ref[:, 3].max() > 0.05   # some pixels see the field
