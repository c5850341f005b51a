"""Incremental rebuild (hdda_grid_update): after an update with the list of
8^3 blocks that may have changed, every array of the grid equals a fresh
build from the new occupancy, bit for bit, and traversal stays equal to the
oracle.  The region map is among the arrays compared.  Covered: changes within partial leaves only (leaves rewritten in
place), changes of block state (empty / partial / full: structure rebuilt),
duplicates and unchanged blocks in the list, the all-blocks form, cascades,
dense grids, and indices outside the grid."""
import numpy as np
import pytest
import torch

from paper_2404_10272_gb300 import scenes
from _helpers import assert_same, gpu_samples, oracle_samples

pytestmark = pytest.mark.gpu

ARRAYS = ("ARRAY_CHILD_MASK", "ARRAY_TILE_MASK", "ARRAY_LEAF_PREFIX", "ARRAY_LEAVES",
          "ARRAY_NODE_SUPER", "ARRAY_LEAF_SUB", "ARRAY_REGION_MAP")


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


def _grid(rng, L, R):
    """Sparse noise, solid boxes (full blocks, tiles) and an empty half."""
    occ = (rng.random((L, R, R, R)) < 0.03).astype(np.uint8)
    for l in range(L):
        for _ in range(3):
            a = rng.integers(0, R - 8, size=3)
            b = np.minimum(a + rng.integers(8, R // 2, size=3), R)
            occ[l, a[0]:b[0], a[1]:b[1], a[2]:b[2]] = 1
        occ[l, : R // 4] = 0
    return occ


def _block_index(L, R, l, bx, by, bz):
    B = (R + 7) // 8
    return l * B ** 3 + (bx * B + by) * B + bz


def _state(blk):
    return 0 if not blk.any() else (2 if blk.all() else 1)


def _edit(rng, occ, kinds):
    """Edits one block per requested kind; returns the new grid and the block list."""
    L, R = occ.shape[0], occ.shape[1]
    B = (R + 7) // 8
    new = occ.copy()
    listed = []
    for kind in kinds:
        for _ in range(10000):
            l = int(rng.integers(0, L))
            bx, by, bz = (int(v) for v in rng.integers(0, B, size=3))
            sl = (l, slice(8 * bx, 8 * bx + 8), slice(8 * by, 8 * by + 8), slice(8 * bz, 8 * bz + 8))
            blk = new[sl]
            st = _state(blk)
            if kind == "partial->partial" and st == 1 and 2 <= blk.sum() <= blk.size - 2:
                ones, zeros = np.argwhere(blk == 1), np.argwhere(blk == 0)
                blk[tuple(ones[0])] = 0
                blk[tuple(zeros[-1])] = 1
            elif kind == "empty->partial" and st == 0:
                blk[0, 0, 0] = 1
            elif kind == "partial->empty" and st == 1:
                blk[...] = 0
            elif kind == "partial->full" and st == 1:
                blk[...] = 1
            elif kind == "full->partial" and st == 2:
                blk[0, 0, 0] = 0
            elif kind == "full->empty" and st == 2:
                blk[...] = 0
            else:
                continue
            listed.append(_block_index(L, R, l, bx, by, bz))
            break
        else:
            raise AssertionError(f"no block for {kind}")
    return new, listed


def _same_as_fresh(H, g, new, aabbs):
    fresh = H.build_vdb(torch.from_numpy(new).cuda(), aabbs)
    for name in ARRAYS:
        which = getattr(H, name)
        np.testing.assert_array_equal(g.array(which), fresh.array(which), err_msg=name)
    a, b = g.stats(), fresh.stats()
    assert (a.n_leaves, a.n_tiles, a.bytes) == (b.n_leaves, b.n_tiles, b.bytes)


def _rays(rng, n):
    o = rng.uniform(-2.5, 2.5, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


@pytest.mark.parametrize("kinds", [
    ["partial->partial"] * 5,                                   # leaves rewritten in place
    ["partial->partial", "empty->partial", "partial->empty"],   # leaf set changes
    ["partial->full", "full->partial", "full->empty", "partial->partial"],  # tiles change
])
def test_update_equals_fresh_build(H, kinds):
    rng = np.random.default_rng(len(kinds) * 7 + 1)
    L, R = 2, 64
    aabbs = scenes.cascade_boxes(L, 1.0)
    occ = _grid(rng, L, R)
    new, listed = _edit(rng, occ, kinds)
    g = H.build_vdb(torch.from_numpy(occ).cuda(), aabbs)
    # an unchanged block and a duplicate ride along
    listed = listed + [listed[0], _block_index(L, R, 0, 0, 0, 0)]
    g.update(torch.from_numpy(new).cuda(), torch.tensor(listed, dtype=torch.int64, device="cuda"))
    _same_as_fresh(H, g, new, aabbs)
    o, d = _rays(rng, 2000)
    p = scenes.SamplerParams(0.0, 6.0, 0.01)
    ref = oracle_samples(o, d, new, aabbs, p)
    prm = H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    assert_same(gpu_samples(H, "hdda", torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                            g, prm), ref, "updated grid")


def test_update_all_blocks_and_repeated_updates(H):
    rng = np.random.default_rng(21)
    L, R = 3, 44                 # R not a multiple of 8 or of 128: edge blocks and nodes
    aabbs = scenes.cascade_boxes(L, 1.0)
    occ = _grid(rng, L, R)
    g = H.build_vdb(torch.from_numpy(occ).cuda(), aabbs)
    cur = occ
    for step in range(4):
        new, listed = _edit(rng, cur, ["partial->partial", "empty->partial", "partial->empty"][: step + 1])
        if step % 2:
            g.update(torch.from_numpy(new).cuda())                      # every block
        else:
            g.update(torch.from_numpy(new).cuda(),
                     torch.tensor(listed, dtype=torch.int64, device="cuda"))
        _same_as_fresh(H, g, new, aabbs)
        cur = new
    # nothing listed: nothing changes
    g.update(torch.from_numpy(cur).cuda(), torch.zeros(0, dtype=torch.int64, device="cuda"))
    _same_as_fresh(H, g, cur, aabbs)


def test_update_with_refinement_off_and_object_scene(H):
    sc = scenes.object_scene()
    rng = np.random.default_rng(5)
    g = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    g.set_refine(False)
    new, listed = _edit(rng, sc.occ, ["partial->partial", "partial->partial", "empty->partial"])
    g.update(torch.from_numpy(new).cuda(), torch.tensor(listed, dtype=torch.int64, device="cuda"))
    g.set_refine(True)
    _same_as_fresh(H, g, new, sc.aabbs)


def test_update_dense_grid_and_bad_indices(H):
    rng = np.random.default_rng(8)
    L, R = 1, 32
    aabbs = scenes.cascade_boxes(L, 1.0)
    occ = _grid(rng, L, R)
    new, listed = _edit(rng, occ, ["empty->partial"])
    gd = H.pack_dense(torch.from_numpy(occ).cuda(), aabbs)
    gd.update(torch.from_numpy(new).cuda(), torch.tensor(listed, dtype=torch.int64, device="cuda"))
    fresh = H.pack_dense(torch.from_numpy(new).cuda(), aabbs)
    np.testing.assert_array_equal(gd.array(H.ARRAY_DENSE_BITS), fresh.array(H.ARRAY_DENSE_BITS))
    g = H.build_vdb(torch.from_numpy(occ).cuda(), aabbs)
    B = (R + 7) // 8
    bad = torch.tensor(listed + [L * B ** 3, -1], dtype=torch.int64, device="cuda")
    with pytest.raises(H.HddaError) as ex:
        g.update(torch.from_numpy(new).cuda(), bad)
    assert ex.value.code == H.ERR_INVALID_ARG
    _same_as_fresh(H, g, new, aabbs)          # the valid entry was applied
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    g.update(torch.from_numpy(new).cuda(), bad, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & (1 << 4)
