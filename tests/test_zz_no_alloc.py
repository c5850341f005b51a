"""The allocation-free hierarchical-DDA entry point.

Some applications cannot let a library allocate GPU memory: they reserve the
whole device up front and hand out fixed buffers, or run loops that must
never enter the CUDA allocator.  hdda_traverse_hdda_noalloc serves them by
keeping its scratch in a fixed device array inside the library.  These tests
call it through the C ABI and check that two calls in a row give exactly the
samples of hdda_traverse_hdda (the suite's bar for samples is bit equality),
and that sizes beyond its fixed limits are refused with a clear error.  Its
own paths are checked against the oracle too: rays with more runs than its
CTAs keep (they walk again and write their own samples) and the largest
single-GPU frame.  The file is named so that pytest runs it after every other
test.
"""
import numpy as np
import pytest
import torch

from paper_2404_10272_gb300 import scenes
from _helpers import assert_same, oracle_samples, slab_scene, subset_rays, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


def _params(H, p):
    return H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)


def _case(H, sc, o, d):
    grid = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    prm = _params(H, sc.params)
    ref = H.traverse_hdda(ot, dt, grid, prm)
    return grid, ot, dt, prm, ref


def test_two_calls_match_allocating_entry_point(H):
    tiny = scenes.tiny_scene()
    o1, d1 = scenes.tiny_camera().rays()
    unb = scenes.unbounded_scene()
    o2, d2 = scenes.unbounded_camera(W=320, H=200).rays()
    for sc, o, d in ((tiny, o1, d1), (unb, o2, d2)):
        grid, ot, dt, prm, ref = _case(H, sc, o, d)
        out = H.alloc_samples(o.shape[0], ref.total + 17)
        out.t0.fill_(float("nan"))
        got = H.traverse_hdda_noalloc(ot, dt, grid, prm, out)
        torch.cuda.synchronize()
        assert got.total == ref.total
        assert_same(tuple(to_np(x) for x in got.trimmed()),
                    tuple(to_np(x) for x in ref.trimmed()), f"noalloc {sc.name}")
    # a second call on the first scene after the array held the second one's data
    grid, ot, dt, prm, ref = _case(H, tiny, o1, d1)
    out = H.alloc_samples(o1.shape[0], ref.total)
    got = H.traverse_hdda_noalloc(ot, dt, grid, prm, out)
    torch.cuda.synchronize()
    assert_same(tuple(to_np(x) for x in got.trimmed()),
                tuple(to_np(x) for x in ref.trimmed()), "noalloc repeat")


def test_limits_are_refused(H):
    sc = scenes.tiny_scene()
    grid = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    prm = _params(H, sc.params)
    n = 2_097_152 + 1
    o = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    d = torch.ones((n, 3), dtype=torch.float32, device="cuda")
    out = H.alloc_samples(n, 1)
    with pytest.raises(H.HddaError) as ex:
        H.traverse_hdda_noalloc(o, d, grid, prm, out)
    assert ex.value.code == H.ERR_INVALID_ARG and "maximum" in str(ex.value)
    # a lattice longer than the fixed table
    o1, d1 = scenes.tiny_camera().rays()
    small = H.alloc_samples(o1.shape[0], 1)
    with pytest.raises(H.HddaError) as ex:
        H.traverse_hdda_noalloc(torch.from_numpy(o1).cuda(), torch.from_numpy(d1).cuda(), grid,
                                H.make_params(0.0, 100.0, 1e-3), small)
    assert ex.value.code == H.ERR_INVALID_ARG and "maximum" in str(ex.value)
    # still usable afterwards
    ref = H.traverse_hdda(torch.from_numpy(o1).cuda(), torch.from_numpy(d1).cuda(), grid, prm)
    out = H.alloc_samples(o1.shape[0], ref.total)
    got = H.traverse_hdda_noalloc(torch.from_numpy(o1).cuda(), torch.from_numpy(d1).cuda(), grid,
                                  prm, out)
    assert got.total == ref.total
    np.testing.assert_array_equal(to_np(got.offsets), to_np(ref.offsets))


def test_rays_with_many_runs_against_oracle(H):
    # Slabs every other voxel: most rays cross more runs than a CTA keeps in shared memory
    # (16), so the one-pass kernel re-walks them and writes their samples itself.  The
    # samples must still be the oracle's, bit for bit, on two calls in a row.
    occ, aabbs, o, d, _, p = slab_scene(128, 2, 700, 7128)
    want = oracle_samples(o, d, occ, aabbs, p)
    off, _, t0, t1 = want
    runs = np.array([1 + int(np.sum(t0[off[r] + 1:off[r + 1]] != t1[off[r]:off[r + 1] - 1]))
                     if off[r + 1] > off[r] else 0 for r in range(o.shape[0])])
    assert (runs > 16).mean() > 0.5
    grid = H.build_vdb(torch.from_numpy(occ).cuda(), aabbs)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    prm = _params(H, p)
    out = H.alloc_samples(o.shape[0], int(off[-1]))
    for call in range(2):
        out.t0.fill_(float("nan"))
        got = H.traverse_hdda_noalloc(ot, dt, grid, prm, out)
        torch.cuda.synchronize()
        assert_same(tuple(to_np(x) for x in got.trimmed()), want, f"many runs, call {call}")


def test_full_unbounded_frame(H):
    # The largest single-GPU frame (4 x 128^3 cascade, 1245 x 825 rays, growing step): all
    # samples equal the allocating sampler's, and a stratified subset of rays (every 97th)
    # equals the oracle's.
    sc = scenes.unbounded_scene()
    o, d = scenes.unbounded_camera().rays()
    grid, ot, dt, prm, ref = _case(H, sc, o, d)
    out = H.alloc_samples(o.shape[0], ref.total)
    got = H.traverse_hdda_noalloc(ot, dt, grid, prm, out)
    torch.cuda.synchronize()
    assert got.total == ref.total
    g_off, g_idx, g_t0, g_t1 = (to_np(x) for x in got.trimmed())
    assert_same((g_off, g_idx, g_t0, g_t1), tuple(to_np(x) for x in ref.trimmed()),
                "noalloc unbounded frame")
    so, sd, sel = subset_rays(o, d, 97, 5)
    want = oracle_samples(so, sd, sc.occ, sc.aabbs, sc.params)
    idx = np.concatenate([np.arange(g_off[r], g_off[r + 1]) for r in sel])
    sub_off = np.concatenate([[0], np.cumsum(g_off[sel + 1] - g_off[sel])])
    sub_idx = np.repeat(np.arange(sel.size, dtype=np.int32), np.diff(sub_off))
    assert np.array_equal(g_idx[idx], np.repeat(sel, np.diff(sub_off)))
    assert_same((sub_off, sub_idx, g_t0[idx], g_t1[idx]), want, "noalloc unbounded subset")
