"""Edge cases at the limits: the most cascade levels, the largest grid (whose tables no longer
fit the shared-memory staging, so the global-memory walk runs), degenerate rays (zero
direction, rays on voxel faces and box faces), all bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_10272_gb300 import scenes
from _helpers import assert_same, gpu_samples, oracle_samples, sampler_form

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


def _check(H, occ, aabbs, o, d, p, what):
    dt = torch.from_numpy(np.ascontiguousarray(occ)).cuda()
    gd, gv = H.pack_dense(dt, aabbs), H.build_vdb(dt, aabbs)
    prm = H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    ot, dd = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    ref = oracle_samples(o, d, occ, aabbs, p)
    assert_same(gpu_samples(H, "dense", ot, dd, gd, prm), ref, what + " dense")
    assert_same(gpu_samples(H, "hdda", ot, dd, gv, prm), ref, what + " hdda")
    gv.set_refine(False)
    assert_same(gpu_samples(H, "hdda", ot, dd, gv, prm), ref, what + " hdda plain")
    with sampler_form(H, H.SAMPLER_FUSED):
        assert_same(gpu_samples(H, "dense", ot, dd, gd, prm), ref, what + " dense fused")
        assert_same(gpu_samples(H, "hdda", ot, dd, gv, prm), ref, what + " hdda plain fused")
    return ref


def _rays(rng, n, spread):
    o = rng.uniform(-spread, spread, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def test_eight_levels(H):
    rng = np.random.default_rng(81)
    L, R = 8, 16
    occ = scenes.random_grid(rng, L, R, 0.15)
    aabbs = scenes.cascade_boxes(L, 0.5)
    o, d = _rays(rng, 1500, 40.0)
    p = scenes.SamplerParams(near=0.0, far=120.0, step=0.05, cone=0.01, max_step=2.0)
    ref = _check(H, occ, aabbs, o, d, p, "L8")
    assert ref[0][-1] > 0


def test_largest_grid(H):
    R = 1024
    occ = np.zeros((1, R, R, R), np.uint8)
    occ[0, 100:140, 200:900, 500:520] = 1          # slabs crossing many nodes
    occ[0, 600:1024, 10:30, 10:30] = 1
    occ[0, 1023, :, 1023] = 1                        # the last voxel plane and row
    rng = np.random.default_rng(1024)
    occ[0][rng.random((R, R, R), dtype=np.float32) < 2e-5] = 1
    aabbs = np.array([[-1.0, -1.0, -1.0, 1.0, 1.0, 1.0]], np.float32)
    o, d = _rays(rng, 600, 1.8)
    p = scenes.SamplerParams(near=0.0, far=5.0, step=2.0 / 1024, cone=0.0)
    ref = _check(H, occ, aabbs, o, d, p, "R1024")
    assert ref[0][-1] > 0


def test_degenerate_rays(H):
    R = 8
    occ = np.zeros((2, R, R, R), np.uint8)
    occ[0, 2:5, 3, 1:7] = 1
    occ[1, :, :, 4] = 1
    aabbs = scenes.cascade_boxes(2, 1.0)
    o = np.array([
        [0.0, 0.0, 0.0],        # zero direction inside an empty voxel of level 0
        [-0.5, -0.125, 0.0],    # zero direction inside an occupied voxel of level 0 (2, 3, 4)
        [-1.0, -0.25, -1.0],    # starts on the lower corner of level 0 (a face of voxel (0, 3, 0))
        [1.0, -0.25, 0.1],      # on the upper x face of level 0: belongs to level 1
        [-3.0, -0.125, 0.125],  # axis-parallel through both levels
        [0.25, 0.25, 5.0],      # outside everything, moving away
        [0.25, 0.25, -5.0],     # outside, entering along z
    ], np.float32)
    d = np.array([
        [0.0, 0.0, 0.0],
        [0.0, -0.0, 0.0],
        [0.0, 0.0, 1.0],
        [-1.0, 0.0, 0.0],
        [1.0, 0.0, 0.0],
        [0.0, 0.0, 1.0],
        [0.0, 0.0, 1.0],
    ], np.float32)
    p = scenes.SamplerParams(near=0.0, far=8.0, step=0.0625)
    ref = _check(H, occ, aabbs, o, d, p, "degenerate")
    cnt = np.diff(ref[0])
    assert cnt[0] == 0 and cnt[1] == 128 and cnt[5] == 0   # all or nothing for zero directions


@pytest.mark.parametrize("form", ["separate", "fused"])
def test_output_alignment_and_capacity_residues(H, form):
    """Sample buffers that are not 16-byte aligned take the element-wise
    emit; capacities of every residue mod 4 end the 16-byte stores exactly at
    capacity on both paths, in both sampler forms."""
    f = H.SAMPLER_FUSED if form == "fused" else H.SAMPLER_SEPARATE
    with sampler_form(H, f):
        _alignment_and_capacity(H)


def _alignment_and_capacity(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    p = sc.params
    prm = H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    full = H.traverse_hdda(ot, dt, g, prm)
    ref = tuple(x.detach().cpu().numpy() for x in full.trimmed())
    assert full.total > 200
    n = o.shape[0]
    for shift in (0, 1, 2, 3):          # element offset of the views: 0 = 16-byte aligned
        for cap in (full.total, full.total - 37, full.total - 38, full.total - 39, full.total - 40):
            buf = H.alloc_samples(n, cap + 8)
            buf.ray_idx.fill_(-7)
            buf.t0.fill_(-1.0)
            buf.t1.fill_(-1.0)
            view = H.Samples(buf.offsets, buf.ray_idx[shift:shift + cap],
                             buf.t0[shift:shift + cap], buf.t1[shift:shift + cap], 0)
            if cap == full.total:
                got = H.traverse_hdda(ot, dt, g, prm, out=view)
                assert_same(tuple(x.detach().cpu().numpy() for x in got.trimmed()), ref,
                            f"shift {shift}")
            else:
                with pytest.raises(H.HddaError) as ex:
                    H.traverse_hdda(ot, dt, g, prm, out=view)
                assert ex.value.code == H.ERR_CAPACITY
                got_t0 = buf.t0[shift:shift + cap].cpu().numpy()
                assert np.array_equal(got_t0.view(np.uint32), ref[2][:cap].view(np.uint32))
                assert np.array_equal(buf.ray_idx[shift:shift + cap].cpu().numpy(), ref[1][:cap])
            # nothing before the view or at or past its capacity
            for arr, fill in ((buf.ray_idx, -7), (buf.t0, -1.0), (buf.t1, -1.0)):
                a = arr.cpu().numpy()
                assert np.all(a[:shift] == fill) and np.all(a[shift + cap:] == fill)
