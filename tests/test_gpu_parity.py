"""GPU parity: dense-grid DDA and hierarchical DDA, called through the C ABI,
against the CPU oracle.  The bar is bit-exact equality of the whole sample
set (offsets, ray indices, t_start and t_end bit patterns)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2404_10272_gb300 import scenes
import _layout
from _helpers import (assert_same, gpu_samples, oracle_samples, sampler_form, slab_scene,
                      subset_rays, to_np)

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_rays.json")


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


def P(H, p):
    return H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)


def both_grids(H, occ, aabbs):
    d = torch.from_numpy(np.ascontiguousarray(occ)).cuda()
    return H.pack_dense(d, aabbs), H.build_vdb(d, aabbs)


def check_all(H, occ, aabbs, o, d, p, what):
    """dense == hdda == oracle, bit-exact."""
    gd, gv = both_grids(H, occ, aabbs)
    prm = P(H, p)
    ref = oracle_samples(o, d, occ, aabbs, p)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    dense = gpu_samples(H, "dense", ot, dt, gd, prm)
    vdb = gpu_samples(H, "hdda", ot, dt, gv, prm)
    assert_same(dense, ref, what + " dense-DDA vs oracle")
    assert_same(vdb, ref, what + " HDDA vs oracle")
    gv.set_refine(False)
    plain = gpu_samples(H, "hdda", ot, dt, gv, prm)
    assert_same(plain, ref, what + " HDDA without refinement vs oracle")
    gv.set_refine(True)
    # Algorithm 2's control flow gives the same samples as Algorithm 1's
    for g, kind in ((gv, "hdda"), (gd, "dense")):
        g.set_walk(H.WALK_SKIP)
        assert_same(gpu_samples(H, kind, ot, dt, g, prm), ref, what + f" {kind} skip form")
        g.set_walk(H.WALK_BRANCH)
    # the walk and the emit fused into one kernel give the same samples
    with sampler_form(H, H.SAMPLER_FUSED):
        assert_same(gpu_samples(H, "dense", ot, dt, gd, prm), ref, what + " dense fused")
        assert_same(gpu_samples(H, "hdda", ot, dt, gv, prm), ref, what + " HDDA fused")
    return ref


with open(GOLDEN) as fh:
    CASES = json.load(fh)["cases"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_worked_rays(H, case):
    L, R = case["levels"], case["res"]
    occ = np.zeros((L, R, R, R), np.uint8)
    if case["occupied"] == "level1_all":
        occ[1] = 1
    else:
        for l, x, y, z in case["occupied"]:
            occ[l, x, y, z] = 1
    o = np.array([case["o"]], np.float32)
    d = np.array([case["d"]], np.float32)
    p = scenes.SamplerParams(case["near"], case["far"], case["step"])
    ref = check_all(H, occ, np.array(case["aabbs"], np.float32), o, d, p, case["name"])
    assert ref[0][-1] == len(case["expect_k"])


def _random_rays(rng, n, spread):
    o = rng.uniform(-spread, spread, size=(n, 3))
    d = rng.normal(size=(n, 3))
    # a quarter of the rays axis-parallel or with zero / negative-zero components
    k = n // 4
    d[:k] = 0.0
    d[np.arange(k), rng.integers(0, 3, size=k)] = rng.choice([-1.0, 1.0], size=k)
    d[k:2 * k, rng.integers(0, 3)] = -0.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # some rays start inside the grid, some far away aimed at it
    o[2 * k:3 * k] *= 0.2
    return o.astype(np.float32), d.astype(np.float32)


def _structured_grid(rng, L, R):
    occ = (rng.random((L, R, R, R)) < 0.05).astype(np.uint8)
    for l in range(L):
        for _ in range(3):  # solid boxes: full 8^3 blocks become tiles, some cross blocks
            a = rng.integers(0, max(1, R - 4), size=3)
            b = np.minimum(a + rng.integers(2, max(3, R // 2), size=3), R)
            occ[l, a[0]:b[0], a[1]:b[1], a[2]:b[2]] = 1
        if l % 2 == 1:
            occ[l, : R // 2] = 0    # a large empty half
    return occ


PROPERTY_CASES = [
    # (levels, res, occupancy kind, cone)
    (1, 5, "bern:0.3", 0.0),
    (1, 16, "struct", 0.0),
    (1, 20, "bern:0.02", 0.0),
    (2, 12, "struct", 0.0),
    (2, 37, "struct", 0.01),
    (3, 24, "bern:0.9", 0.0),
    (4, 16, "struct", 0.004),
    (4, 32, "struct", 0.05),
    (1, 64, "empty", 0.0),
    (2, 8, "full", 0.0),
    (1, 136, "struct", 0.0),      # more than one 16^3-block node per axis
]


@pytest.mark.parametrize("levels,res,kind,cone", PROPERTY_CASES)
def test_property_cases(H, levels, res, kind, cone):
    rng = np.random.default_rng(levels * 1000 + res)
    if kind.startswith("bern"):
        occ = scenes.random_grid(rng, levels, res, float(kind.split(":")[1]))
    elif kind == "struct":
        occ = _structured_grid(rng, levels, res)
    elif kind == "empty":
        occ = np.zeros((levels, res, res, res), np.uint8)
    else:
        occ = np.ones((levels, res, res, res), np.uint8)
    aabbs = scenes.cascade_boxes(levels, 0.8)
    if levels == 1:
        aabbs = np.array([[-0.8, -0.7, -0.9, 0.8, 0.75, 0.6]], np.float32)  # non-cubic box
    n = 3000 if res <= 64 else 600
    o, d = _random_rays(rng, n, 2.5)
    p = scenes.SamplerParams(near=0.0, far=7.0, step=0.0123, cone=cone)
    check_all(H, occ, aabbs, o, d, p, f"L{levels} R{res} {kind}")


# Lattices of every shape the walk's first guess of a crossing index treats differently:
# constant spacing (no growth, or a cap below the step), a constant start then geometric
# growth (from inside the lattice, from its first index, or never reached), and a growth the
# cap max_step ends (the bucket index).  (near, far, step, cone, max_step)
LATTICES = [
    (0.0, 7.0, 0.0123, 0.0, 1e10),    # constant step
    (0.0, 7.0, 0.01, 0.02, 0.005),    # cap below the step: constant max_step
    (0.0, 7.0, 0.0123, 0.05, 1e10),   # constant, then geometric from t = 0.246
    (1.0, 7.0, 0.01, 0.05, 1e10),     # geometric from the first index
    (0.0, 7.0, 0.05, 0.002, 1e10),    # growth never reached
    (0.0, 20.0, 0.01, 0.05, 0.2),     # geometric, then capped from t = 4
]


@pytest.mark.parametrize("lattice", LATTICES, ids=[f"lattice{i}" for i in range(len(LATTICES))])
def test_lattice_shapes(H, lattice):
    """The samplers stay bit-exact whichever way the crossing search guesses its indices."""
    near, far, step, cone, max_step = lattice
    rng = np.random.default_rng(4242)
    occ = _structured_grid(rng, 2, 24)
    aabbs = scenes.cascade_boxes(2, 0.8)
    o, d = _random_rays(rng, 800, 2.5)
    p = scenes.SamplerParams(near=near, far=far, step=step, cone=cone, max_step=max_step)
    ref = check_all(H, occ, aabbs, o, d, p, f"lattice {lattice}")
    assert ref[0][-1] > 0


@pytest.mark.parametrize("R,period", [(64, 2), (128, 3)])
def test_rays_with_many_runs(H, R, period):
    """Rays crossing more occupied slabs than the walk keeps runs for (16)
    walk again in the emit and write their own samples; tiles mix them with
    rays of a few runs (every third ray turned to run along the slabs)."""
    occ, aabbs, o, d, _, p = slab_scene(R, period, 900, 5000 + R + period)
    o, d = o.copy(), d.astype(np.float64)
    # every third ray starts in slab 0 and runs nearly along the slabs: 1 to a few runs
    o[::3, 0] = 0.5 / R
    m = o[::3].shape[0]
    d[::3] = np.stack([np.linspace(0.0, 0.08, m), np.full(m, 0.6), np.full(m, 0.8)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = d.astype(np.float32)
    ref = check_all(H, occ, aabbs, o, d, p, f"slabs R{R} period {period}")

    def n_runs(r):
        a, b = ref[0][r], ref[0][r + 1]
        return 0 if a == b else 1 + int(np.count_nonzero(ref[2][a + 1:b] != ref[3][a:b - 1]))

    runs = np.array([n_runs(r) for r in range(o.shape[0])])
    assert (runs[1::3] > 16).mean() > 0.9   # most rays across the slabs overflow the 16 kept runs
    assert 1 <= runs[::3].min() and runs[::3].max() <= 16


def test_tiny_scene_full_frame(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    ref = check_all(H, sc.occ, sc.aabbs, o, d, sc.params, "tiny 96x96")
    assert ref[0][-1] > 0


def _full_vs_subset(H, sc, o, d, width, stride, what):
    gd, gv = both_grids(H, sc.occ, sc.aabbs)
    prm = P(H, sc.params)
    p = sc.params
    # the launch the benchmark times: the image width passed (8 x 4 pixel blocks)
    prm_w = H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps,
                          image_width=width)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    dense = gpu_samples(H, "dense", ot, dt, gd, prm)
    vdb = gpu_samples(H, "hdda", ot, dt, gv, prm)
    assert_same(dense, vdb, what + " full frame: dense-DDA vs HDDA")
    gv.set_refine(False)
    assert_same(gpu_samples(H, "hdda", ot, dt, gv, prm), vdb, what + " full frame: plain vs refined")
    gv.set_refine(True)
    # the library default (region checks off) and the image width, as the benchmark runs it
    H.set_region_checks(False)
    try:
        assert_same(gpu_samples(H, "hdda", ot, dt, gv, prm), vdb, what + " full frame: checks off")
        assert_same(gpu_samples(H, "dense", ot, dt, gd, prm), dense,
                    what + " full frame: dense, checks off")
        timed = gpu_samples(H, "hdda", ot, dt, gv, prm_w)
        assert_same(timed, vdb, what + " full frame: pixel blocks, checks off")
        assert_same(gpu_samples(H, "dense", ot, dt, gd, prm_w), dense,
                    what + " full frame: dense, pixel blocks, checks off")
    finally:
        H.set_region_checks(True)
    with sampler_form(H, H.SAMPLER_FUSED):
        assert_same(gpu_samples(H, "hdda", ot, dt, gv, prm), vdb, what + " full frame: fused")
        assert_same(gpu_samples(H, "dense", ot, dt, gd, prm), dense,
                    what + " full frame: dense, fused")
    # oracle on a stratified subset of the timed launch's rays
    so, sd, sel = subset_rays(o, d, stride, offset=stride // 3)
    ref = oracle_samples(so, sd, sc.occ, sc.aabbs, sc.params)
    off, idx, t0, t1 = timed
    for j, r in enumerate(sel):
        a, b = off[r], off[r + 1]
        ra, rb = ref[0][j], ref[0][j + 1]
        assert b - a == rb - ra, (what, r)
        assert np.all(idx[a:b] == r)
        assert np.array_equal(t0[a:b].view(np.uint32), ref[2][ra:rb].view(np.uint32)), (what, r)
        assert np.array_equal(t1[a:b].view(np.uint32), ref[3][ra:rb].view(np.uint32)), (what, r)
    return vdb


def test_object_scene_full_size(H):
    sc = scenes.object_scene()
    o, d = scenes.object_cameras(n=1)[0].rays()
    vdb = _full_vs_subset(H, sc, o, d, 800, 97, "object 800x800")
    assert vdb[0][-1] > 1_000_000


def test_unbounded_scene_full_size(H):
    sc = scenes.unbounded_scene()
    o, d = scenes.unbounded_camera().rays()
    vdb = _full_vs_subset(H, sc, o, d, 1245, 211, "unbounded 1245x825")
    assert vdb[0][-1] > 0


def test_grid_structures_match_oracle(H):
    rng = np.random.default_rng(5)
    occ = _structured_grid(rng, 3, 37)
    aabbs = scenes.cascade_boxes(3, 1.0)
    gd, gv = both_grids(H, occ, aabbs)
    words = oracle.pack_dense_bits(occ)
    np.testing.assert_array_equal(gd.array(H.ARRAY_DENSE_BITS), words.reshape(-1))
    v = oracle.build_vdb(occ)
    np.testing.assert_array_equal(gv.array(H.ARRAY_CHILD_MASK), v["child"].reshape(-1))
    np.testing.assert_array_equal(gv.array(H.ARRAY_TILE_MASK), v["tile"].reshape(-1))
    np.testing.assert_array_equal(gv.array(H.ARRAY_LEAVES), v["leaves"].reshape(-1))
    st = gv.stats()
    assert st.n_leaves == v["n_leaves"] and st.n_tiles == v["n_tiles"]
    assert st.dense_bytes == 3 * oracle.dense_words_per_level(37) * 4
    nsuper, lsub = _layout.vdb_refinement(v)
    np.testing.assert_array_equal(gv.array(H.ARRAY_NODE_SUPER), nsuper.reshape(-1))
    np.testing.assert_array_equal(gv.array(H.ARRAY_LEAF_SUB), lsub.reshape(-1))
    # region map (R = 37: odd, so the last cell per axis holds one voxel and padding)
    np.testing.assert_array_equal(gv.array(H.ARRAY_REGION_MAP), _layout.region_map(occ).reshape(-1))
    assert st.map_bytes == 3 * 19 ** 3 * 2
    # leaf prefix: global index of the first leaf of each child-mask word
    child = v["child"].reshape(-1)
    pc = np.array([bin(int(w)).count("1") for w in child])
    np.testing.assert_array_equal(gv.array(H.ARRAY_LEAF_PREFIX),
                                  np.concatenate([[0], np.cumsum(pc)[:-1]]))


def test_thresholds_are_exact_voxel_boundaries(H):
    sc = scenes.object_scene()
    g = H.pack_dense(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    R = sc.res
    thr = g.array(H.ARRAY_THRESHOLDS).reshape(1, 3, R + 1)
    f32 = np.float32
    for c in range(3):
        lo, hi = f32(sc.aabbs[0, c]), f32(sc.aabbs[0, 3 + c])
        s = f32(R) / f32(hi - lo)
        X = thr[0, c]
        assert X[0] == lo and X[R] == hi
        idx = lambda x: min(max(int(np.floor(f32(f32(x - lo) * s))), 0), R - 1)
        for a in range(1, R):
            assert idx(X[a]) >= a
            assert idx(np.nextafter(X[a], f32(-np.inf))) < a


def test_table3_sizes(H):
    """Dense 128^3 bit array = 256 KiB (Table 3 caption); the VDB is reported beside it."""
    sc = scenes.object_scene()
    gd, gv = both_grids(H, sc.occ, sc.aabbs)
    assert gd.stats().dense_bytes == 256 * 1024
    st = gv.stats()
    v = oracle.build_vdb(sc.occ)
    assert st.n_leaves == v["n_leaves"] and st.n_tiles == v["n_tiles"]
    # level table + thresholds + node masks + leaves + refinement masks (18 words per
    # node, 5 per leaf)
    assert st.bytes == (36 + 3 * 129 * 4 + (3 * 128 * 4 + 4) + 64 * v["n_leaves"]
                        + 18 * 4 + 20 * v["n_leaves"])
    gv.set_refine(False)
    assert gv.stats().bytes == 36 + 3 * 129 * 4 + (3 * 128 * 4 + 4) + 64 * v["n_leaves"]
    # the region map beside it: 2 bytes per 2^3 cell, twice the dense bit array
    assert st.map_bytes == 2 * 64 ** 3 == 2 * gd.stats().dense_bytes


def test_rebuild_matches_fresh_build(H):
    rng = np.random.default_rng(9)
    occ_a = _structured_grid(rng, 2, 32)
    occ_b = _structured_grid(rng, 2, 32)
    aabbs = scenes.cascade_boxes(2, 1.0)
    gd, gv = both_grids(H, occ_a, aabbs)
    db = torch.from_numpy(occ_b).cuda()
    gd.rebuild(db)
    gv.rebuild(db)
    o, d = _random_rays(rng, 1000, 2.5)
    p = scenes.SamplerParams(0.0, 6.0, 0.01)
    ref = oracle_samples(o, d, occ_b, aabbs, p)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    assert_same(gpu_samples(H, "dense", ot, dt, gd, P(H, p)), ref, "rebuilt dense")
    assert_same(gpu_samples(H, "hdda", ot, dt, gv, P(H, p)), ref, "rebuilt vdb")


def test_batch_split_and_permutation_invariance(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    _, gv = both_grids(H, sc.occ, sc.aabbs)
    prm = P(H, sc.params)
    whole = gpu_samples(H, "hdda", torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), gv, prm)
    perm = np.random.default_rng(3).permutation(o.shape[0])
    parts = [perm[:1000], perm[1000:1001], perm[1001:]]
    for part in parts:
        po, pd = torch.from_numpy(o[part]).cuda(), torch.from_numpy(d[part]).cuda()
        off, idx, t0, t1 = gpu_samples(H, "hdda", po, pd, gv, prm)
        for j, r in enumerate(part):
            a, b = whole[0][r], whole[0][r + 1]
            assert np.array_equal(t0[off[j]:off[j + 1]].view(np.uint32), whole[2][a:b].view(np.uint32))
            assert np.all(idx[off[j]:off[j + 1]] == j)


def test_edge_cases(H):
    sc = scenes.tiny_scene()
    gd, gv = both_grids(H, sc.occ, sc.aabbs)
    o, d = scenes.tiny_camera().rays()
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    prm = P(H, sc.params)
    # no rays
    e = H.traverse_hdda(ot[:0], dt[:0], gv, prm)
    assert e.total == 0 and to_np(e.offsets).tolist() == [0]
    # empty lattice (near beyond far)
    s = H.traverse_hdda(ot, dt, gv, H.make_params(7.0, 6.0, 0.01))
    assert s.total == 0 and not to_np(s.offsets).any()
    # count only fills CSR offsets
    c = H.traverse_dense(ot, dt, gd, prm, count_only=True)
    full = H.traverse_dense(ot, dt, gd, prm)
    assert c.total == full.total
    np.testing.assert_array_equal(to_np(c.offsets), to_np(full.offsets))
    # capacity below the total is an error that writes nothing at or past capacity
    cap = max(1, full.total - 100)
    big = H.alloc_samples(o.shape[0], full.total)
    for t in (big.t0, big.t1):
        t.fill_(-1.0)
    big.ray_idx.fill_(-7)
    small = H.Samples(big.offsets, big.ray_idx[:cap], big.t0[:cap], big.t1[:cap], 0)
    with pytest.raises(H.HddaError) as ex:
        H.traverse_hdda(ot, dt, gv, prm, out=small)
    assert ex.value.code == H.ERR_CAPACITY
    assert small.total == full.total
    assert bool((big.t0[cap:] == -1.0).all()) and bool((big.ray_idx[cap:] == -7).all())
    # what was written below capacity is the true prefix of the sample set
    np.testing.assert_array_equal(to_np(big.t0[:cap]), to_np(full.t0[:cap]))
    # more candidates than max_steps
    with pytest.raises(H.HddaError) as ex:
        H.traverse_hdda(ot, dt, gv, H.make_params(2.0, 6.0, 5e-3, max_steps=100))
    assert ex.value.code == H.ERR_STEP_LIMIT
    # invalid parameters and wrong grid kind
    for bad in [H.make_params(2.0, 6.0, 0.0), H.make_params(2.0, float("inf"), 0.01),
                H.make_params(2.0, 6.0, 0.01, cone=-1.0)]:
        with pytest.raises(H.HddaError) as ex:
            H.traverse_hdda(ot, dt, gv, bad)
        assert ex.value.code == H.ERR_INVALID_ARG
    with pytest.raises(H.HddaError):
        H.traverse_hdda(ot, dt, gd, prm)
    with pytest.raises(H.HddaError):
        H.traverse_dense(ot, dt, gv, prm)
    # non-finite rays have no samples; their neighbours are unaffected
    o2, d2 = o.copy(), d.copy()
    o2[5, 0] = np.nan
    d2[7, 1] = np.inf
    s2 = H.traverse_hdda(torch.from_numpy(o2).cuda(), torch.from_numpy(d2).cuda(), gv, prm)
    cnt2 = np.diff(to_np(s2.offsets))
    cnt = np.diff(to_np(full.offsets))
    assert cnt2[5] == 0 and cnt2[7] == 0
    keep = np.ones(o.shape[0], bool)
    keep[[5, 7]] = False
    np.testing.assert_array_equal(cnt2[keep], cnt[keep])
    # invalid grid construction
    with pytest.raises(H.HddaError):
        H.build_vdb(torch.zeros((1, 4, 4, 4), dtype=torch.uint8, device="cuda"),
                    [[0, 0, 0, 1, 0, 1]])
