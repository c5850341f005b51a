"""Pins of the CPU oracle against facts fixed independently of it.

Each pin is chosen so that a plausible slip in the oracle fails at least one:
hand-worked dyadic rays (midpoint rule, half-open voxels and boxes, finer
cascade level wins, axis order, direction sign), the binary32 recurrence
(0.1f summed ten times), the min/max order of the step clamp, the index
clamp just below the box's upper face, float64 geometry away from
boundaries, complement and permutation invariants, closed-form compositing
and the dense/VDB storage facts of Table 3.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2404_10272_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_rays.json")
f32 = np.float32


def _grid_from_case(case):
    L, R = case["levels"], case["res"]
    occ = np.zeros((L, R, R, R), np.uint8)
    if case["occupied"] == "level1_all":
        occ[1] = 1
    else:
        for l, x, y, z in case["occupied"]:
            occ[l, x, y, z] = 1
    return occ


def _run_case(case, **kw):
    occ = _grid_from_case(case)
    o = np.array([case["o"]], np.float32)
    d = np.array([case["d"]], np.float32)
    return oracle.sample(o, d, occ, case["aabbs"], case["near"], case["far"], case["step"], 0.0,
                         **kw)


with open(GOLDEN) as fh:
    CASES = json.load(fh)["cases"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_worked_rays(case):
    off, idx, t0, t1 = _run_case(case)
    lat = oracle.lattice(case["near"], case["far"], case["step"])
    assert lat.size - 1 == case["candidates"]
    ks = [int(np.flatnonzero(lat == a)[0]) for a in t0]
    assert ks == case["expect_k"]
    assert np.all(idx == 0)
    assert off.tolist() == [0, len(case["expect_k"])]
    if "expect_t" in case:
        np.testing.assert_array_equal(np.stack([t0, t1], -1).reshape(-1, 2),
                                      np.array(case["expect_t"], np.float32).reshape(-1, 2))
    # every kept interval is one lattice step
    for a, b in zip(t0, t1):
        k = int(np.flatnonzero(lat == a)[0])
        assert lat[k + 1] == b


def test_recurrence_not_closed_form():
    # 0.1f added ten times is 1.0000001f in binary32, while 10 * 0.1f is 1.0f.
    lat = oracle.lattice(0.0, 1.5, 0.1)
    assert lat[10] == f32(1.0000001)
    assert lat[10] != f32(1.0)
    assert f32(10) * f32(0.1) == f32(1.0)


def test_linear_step_growth_and_clamp_order():
    # cone 1 doubles t exactly: 1, 2, 4, 8
    np.testing.assert_array_equal(oracle.lattice(1.0, 8.0, 0.25, cone=1.0), [1, 2, 4, 8])
    # max_step caps the growth: 1, 2, 4, 6, 8
    np.testing.assert_array_equal(oracle.lattice(1.0, 8.0, 0.25, cone=1.0, max_step=2.0),
                                  [1, 2, 4, 6, 8])
    # min(max(t*cone, step), max_step): a max_step below step wins (0, 2, 4, 6, 8);
    # the other nesting would give 0, 3, 6
    np.testing.assert_array_equal(oracle.lattice(0.0, 8.0, 3.0, cone=0.0, max_step=2.0),
                                  [0, 2, 4, 6, 8])
    # the step stays constant while t * cone <= step, then grows: 0.75 * 0.5 = 0.375
    np.testing.assert_array_equal(oracle.lattice(0.0, 1.2, 0.25, cone=0.5),
                                  [0, 0.25, 0.5, 0.75, 1.125])


def test_stop_rule_keeps_last_candidate_reaching_far():
    # t_{k+1} <= far keeps the candidate ending exactly at far
    assert oracle.lattice(0.0, 1.0, 0.25).tolist() == [0, 0.25, 0.5, 0.75, 1.0]
    assert oracle.lattice(0.0, 0.99, 0.25).tolist() == [0, 0.25, 0.5, 0.75]
    assert oracle.lattice(2.0, 1.0, 0.25).tolist() == [2.0]


def test_step_limit_is_an_error():
    case = CASES[0]
    with pytest.raises(oracle.OracleError) as e:
        _run_case(case, max_steps=31)
    assert e.value.code == oracle.ERR_STEP_LIMIT
    off, *_ = _run_case(case, max_steps=32)
    assert off[-1] == 4


def test_invalid_params_rejected():
    o = np.zeros((1, 3), np.float32)
    occ = np.ones((1, 2, 2, 2), np.uint8)
    box = [0, 0, 0, 1, 1, 1]
    for bad in [dict(step=0.0), dict(step=-1.0), dict(cone=-0.1), dict(far=math.inf),
                dict(near=math.nan)]:
        kw = dict(near=0.0, far=1.0, step=0.1, cone=0.0)
        kw.update(bad)
        with pytest.raises(oracle.OracleError):
            oracle.sample(o, o, occ, box, kw["near"], kw["far"], kw["step"], kw["cone"])
    with pytest.raises(oracle.OracleError):
        oracle.sample(o, o, occ, [0, 0, 0, 1, 0, 1], 0.0, 1.0, 0.1)  # hi == lo


def test_index_clamped_below_upper_face():
    # x = nextafter(1.5, 0) over [-1.5, 1.5) with R = 128: (x + 1.5) rounds to 3.0 and
    # 3.0 * fl(128/3) rounds to 128.0, so the voxel index must clamp to 127.
    x = np.nextafter(f32(1.5), f32(0))
    s = f32(128) / f32(3.0)
    assert np.floor(f32(f32(x + f32(1.5)) * s)) == 128.0
    occ = np.zeros((1, 128, 128, 128), np.uint8)
    occ[0, 127] = 1
    o = np.array([[x, -2.0, 0.1]], np.float32)
    d = np.array([[0.0, 1.0, 0.0]], np.float32)
    off, idx, t0, t1 = oracle.sample(o, d, occ, [-1.5] * 3 + [1.5] * 3, 0.0, 4.0, 1.0 / 64)
    # y = -2 + (2k+1)/128 is inside [-1.5, 1.5) for k = 32 .. 223
    assert off[-1] == 192
    assert t0[0] == f32(32 / 64) and t1[-1] == f32(224 / 64)
    # one ulp further down the plane x = 127 is not reached at all by a wrong clamp
    occ2 = np.zeros_like(occ)
    occ2[0, 126] = 1
    off2, *_ = oracle.sample(o, d, occ2, [-1.5] * 3 + [1.5] * 3, 0.0, 4.0, 1.0 / 64)
    assert off2[-1] == 0


def test_empty_and_full_grids_and_nonfinite_rays():
    rng = np.random.default_rng(7)
    o = rng.uniform(-2, 2, size=(64, 3)).astype(np.float32)
    d = rng.normal(size=(64, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    box = [-1, -1, -1, 1, 1, 1]
    off, *_ = oracle.sample(o, d, np.zeros((1, 8, 8, 8), np.uint8), box, 0.0, 4.0, 0.01)
    assert off[-1] == 0
    o[3, 1] = np.nan
    d[5, 2] = np.inf
    off, idx, t0, t1 = oracle.sample(o, d, np.ones((1, 8, 8, 8), np.uint8), box, 0.0, 4.0, 0.01)
    cnt = np.diff(off)
    assert cnt[3] == 0 and cnt[5] == 0
    # full single level: kept == candidates whose midpoint lies in the box (float64 check
    # away from the faces)
    lat = oracle.lattice(0.0, 4.0, 0.01).astype(np.float64)
    tm = 0.5 * (lat[:-1] + lat[1:])
    for r in range(64):
        if r in (3, 5):
            continue
        x = o[r].astype(np.float64)[None] + tm[:, None] * d[r].astype(np.float64)[None]
        inside = np.all((x >= -1) & (x < 1), axis=1)
        margin = np.min(np.minimum(np.abs(x + 1), np.abs(x - 1)), axis=1)
        clear = margin > 1e-5
        got = np.zeros(tm.size, bool)
        ks = np.searchsorted(lat, t0[off[r]:off[r + 1]].astype(np.float64))
        got[ks] = True
        assert np.array_equal(got[clear], inside[clear])


def _locate64(x, occ, aabbs):
    """float64 geometric point location: (occupied, distance to the nearest face)."""
    L, R = occ.shape[0], occ.shape[1]
    best = math.inf
    for l in range(L):
        lo, hi = np.float64(aabbs[l][:3]), np.float64(aabbs[l][3:])
        u = (x - lo) / (hi - lo) * R
        best = min(best, float(np.min(np.abs(u - np.round(u)))) / R * float(np.min(hi - lo)))
        if np.all((x >= lo) & (x < hi)):
            i = np.minimum(np.floor(u).astype(int), R - 1)
            return bool(occ[l, i[0], i[1], i[2]]), best
    return False, best


@pytest.mark.parametrize("levels,res,cone", [(1, 5, 0.0), (2, 6, 0.0), (3, 4, 0.05), (4, 8, 0.004)])
def test_float64_geometry_away_from_faces(levels, res, cone):
    """Every candidate whose midpoint is clearly inside one voxel is classified the way
    float64 geometry says; only points within 1e-5 of a face may go either way."""
    rng = np.random.default_rng(100 + levels * 10 + res)
    occ = scenes.random_grid(rng, levels, res, 0.4)
    aabbs = scenes.cascade_boxes(levels, 0.75)
    n = 48
    o = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    near, far, step = 0.0, 6.0, 0.02
    off, idx, t0, t1 = oracle.sample(o, d, occ, aabbs, near, far, step, cone)
    lat = oracle.lattice(near, far, step, cone).astype(np.float64)
    tm = 0.5 * (lat[:-1] + lat[1:])
    checked = 0
    for r in range(n):
        kept = np.zeros(tm.size, bool)
        kept[np.searchsorted(lat, t0[off[r]:off[r + 1]].astype(np.float64))] = True
        for k in range(tm.size):
            x = o[r].astype(np.float64) + tm[k] * d[r].astype(np.float64)
            occd, margin = _locate64(x, occ, aabbs)
            if margin > 1e-5:
                assert kept[k] == occd, (r, k)
                checked += 1
    assert checked > 0.9 * n * tm.size


def test_complement_and_permutation_invariants():
    rng = np.random.default_rng(11)
    L, R = 2, 12
    occ = scenes.random_grid(rng, L, R, 0.3)
    aabbs = scenes.cascade_boxes(L, 0.6)
    n = 40
    o = rng.uniform(-1.5, 1.5, size=(n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    args = (0.0, 5.0, 0.013, 0.01)
    a = oracle.sample(o, d, occ, aabbs, *args)
    b = oracle.sample(o, d, 1 - occ, aabbs, *args)
    f = oracle.sample(o, d, np.ones_like(occ), aabbs, *args)
    for r in range(n):
        sa = set(a[2][a[0][r]:a[0][r + 1]].tolist())
        sb = set(b[2][b[0][r]:b[0][r + 1]].tolist())
        sf = set(f[2][f[0][r]:f[0][r + 1]].tolist())
        assert not (sa & sb)
        assert sa | sb == sf
        seg = f[2][f[0][r]:f[0][r + 1]]
        assert np.all(np.diff(seg) > 0)
        # consecutive kept steps share their end point
        t0s, t1s = f[2][f[0][r]:f[0][r + 1]], f[3][f[0][r]:f[0][r + 1]]
        lat = oracle.lattice(*args)
        for j in range(len(t0s) - 1):
            k = int(np.flatnonzero(lat == t0s[j])[0])
            if lat[k + 1] == t0s[j + 1]:
                assert t1s[j] == t0s[j + 1]
    perm = rng.permutation(n)
    p = oracle.sample(o[perm], d[perm], occ, aabbs, *args)
    for new, old in enumerate(perm):
        np.testing.assert_array_equal(p[2][p[0][new]:p[0][new + 1]], a[2][a[0][old]:a[0][old + 1]])
        assert np.all(p[1][p[0][new]:p[0][new + 1]] == new)


def test_composite_closed_forms():
    # one blob with a huge radius is a constant field: sigma = a, colour = rgb, and the
    # product of transmittances telescopes to exp(-a * sum(dt)).
    field = np.array([[0, 0, 0, 1e6, 3.0, 0.2, 0.5, 0.9]], np.float32)
    o = np.zeros((3, 3), np.float32)
    d = np.tile(np.array([[1, 0, 0]], np.float32), (3, 1))
    t0 = np.array([0.0, 0.25, 0.5, 1.0, 2.0], np.float32)
    t1 = np.array([0.25, 0.5, 0.75, 1.5, 2.125], np.float32)
    off = np.array([0, 0, 1, 5], np.int64)
    rgba = oracle.composite(o, d, off, t0, t1, field)
    np.testing.assert_array_equal(rgba[0], [0, 0, 0, 0])       # no samples
    c = field[0, 5:8].astype(np.float64)                        # float32-rounded colour
    a1 = 1 - math.exp(-3.0 * 0.25)                              # one sample: alpha * c
    np.testing.assert_allclose(rgba[1], [*(a1 * c), a1], rtol=1e-9)
    tot = 0.25 + 0.25 + 0.5 + 0.125
    a = 1 - math.exp(-3.0 * tot)
    np.testing.assert_allclose(rgba[2], [*(a * c), a], rtol=1e-9)


def test_composite_front_to_back_order():
    # two disjoint blobs of different colour: the nearer one is weighted by T = 1,
    # the farther by the transmittance left after the first.
    field = np.array([[1, 0, 0, 0.05, 40.0, 1, 0, 0], [3, 0, 0, 0.05, 40.0, 0, 0, 1]], np.float32)
    o = np.zeros((1, 3), np.float32)
    d = np.array([[1, 0, 0]], np.float32)
    t0 = np.array([0.9, 2.9], np.float32)
    t1 = np.array([1.1, 3.1], np.float32)
    rgba = oracle.composite(o, d, np.array([0, 2], np.int64), t0, t1, field)[0]
    s = 40.0  # at the blob centres the other blob is 2 away: exp(-2^2/(2*0.05^2)) underflows
    a = 1 - math.exp(-s * (np.float64(t1[0]) - np.float64(t0[0])))
    b = 1 - math.exp(-s * (np.float64(t1[1]) - np.float64(t0[1])))
    np.testing.assert_allclose(rgba, [a, 0, (1 - a) * b, 1 - (1 - a) * (1 - b)], rtol=1e-12)


def test_dense_bits_layout_and_size():
    R = 4
    occ = np.zeros((2, R, R, R), np.uint8)
    occ[0, 0, 0, 1] = 1     # linear 1
    occ[0, 1, 0, 0] = 1     # linear 16
    occ[1, 3, 3, 3] = 1     # linear 63 of level 1
    w = oracle.pack_dense_bits(occ)
    assert w.shape == (2, 2)
    assert w[0, 0] == (1 << 1) | (1 << 16) and w[0, 1] == 0
    assert w[1, 1] == (1 << 31)
    # Table 3 caption: one 128^3 grid is 256 KiB as a bit array, four are 1024 KiB
    assert oracle.dense_words_per_level(128) * 4 == 256 * 1024
    assert 4 * oracle.dense_words_per_level(128) * 4 == 1024 * 1024


@pytest.mark.parametrize("res,p", [(20, 0.3), (16, 0.0), (8, 1.0), (37, 0.02)])
def test_vdb_round_trip_and_counts(res, p):
    rng = np.random.default_rng(res)
    occ = scenes.random_grid(rng, 2, res, p)
    if res == 37:
        occ[1, :16, :16, :16] = 1      # two full blocks plus partial edges
    v = oracle.build_vdb(occ)
    assert np.array_equal(oracle.densify_vdb(v), occ)
    # leaf and tile counts by direct slicing of each block
    B = (res + 7) // 8
    partial = full = 0
    for l in range(2):
        for bx in range(B):
            for by in range(B):
                for bz in range(B):
                    blk = occ[l, bx * 8:bx * 8 + 8, by * 8:by * 8 + 8, bz * 8:bz * 8 + 8]
                    s = int(blk.sum())
                    if s == 512:
                        full += 1
                    elif s > 0:
                        partial += 1
    assert v["n_leaves"] == partial and v["n_tiles"] == full
    # tile and child bits never overlap
    assert not np.any(v["child"] & v["tile"])


def _one_sample(field, o, d, t0, t1):
    o = np.array([o], np.float32)
    d = np.array([d], np.float32)
    return oracle.composite(o, d, np.array([0, 1], np.int64), np.array([t0], np.float32),
                            np.array([t1], np.float32), np.array(field, np.float32))[0]


@pytest.mark.parametrize("o,dist2", [
    ((-1.0, 0.5, 0.0), 0.25),      # midpoint (0, 0.5, 0): one radius off the centre
    ((-1.0, 1.0, 0.0), 1.0),       # (0, 1, 0): two radii
    ((-1.5, 0.0, 0.0), 0.25),      # (-0.5, 0, 0): one radius along the ray's own axis
    ((-0.75, 0.25, 0.25), 0.1875),  # (0.25, 0.25, 0.25): all three components
])
def test_composite_gaussian_falloff(o, dist2):
    # One blob of amplitude a and radius s at the origin, one interval [0.75, 1.25] along +x
    # whose midpoint (t = 1) lies at squared distance dist2 from the centre: the density is
    # a * exp(-dist2 / (2 s^2)) (Sec. 1's field; the Gaussian's 2 s^2), the colour the blob's
    # own, and the pixel (1 - exp(-sigma * dt)) * rgb with dt = 0.5.  Every input and the
    # midpoint are exact in binary32.
    a, s, rgb = 4.0, 0.5, np.array([0.25, 0.5, 0.75])
    px = _one_sample([[0, 0, 0, s, a, *rgb]], o, (1, 0, 0), 0.75, 1.25)
    sigma = a * math.exp(-dist2 / (2 * s * s))
    alpha = 1 - math.exp(-sigma * 0.5)
    np.testing.assert_allclose(px, [*(alpha * rgb), alpha], rtol=1e-12)


def test_composite_colour_is_density_weighted_mean():
    # Two blobs seen from one point at different distances: weights w1 = a1 e^(-1/2) (one
    # radius) and w2 = a2 e^(-2) (two radii).  The density is w1 + w2 and the colour the
    # density-weighted mean (w1 rgb1 + w2 rgb2) / (w1 + w2), not the plain mean of the two.
    rgb1, rgb2 = np.array([1.0, 0.0, 0.5]), np.array([0.0, 1.0, 0.25])
    field = [[0, 0, 0, 0.5, 2.0, *rgb1], [0, 1.5, 0, 0.5, 3.0, *rgb2]]
    px = _one_sample(field, (-1, 0.5, 0), (1, 0, 0), 0.75, 1.25)   # midpoint (0, 0.5, 0)
    w1, w2 = 2.0 * math.exp(-0.5), 3.0 * math.exp(-2.0)
    colour = (w1 * rgb1 + w2 * rgb2) / (w1 + w2)
    alpha = 1 - math.exp(-(w1 + w2) * 0.5)
    np.testing.assert_allclose(px, [*(alpha * colour), alpha], rtol=1e-12)
    # the plain mean differs by far more than the tolerance
    assert np.abs(alpha * (rgb1 + rgb2) / 2 - px[:3]).max() > 0.05
