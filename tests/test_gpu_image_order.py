"""Ray-order hint (hdda_params.image_width): when the rays are the pixels of a
W-wide image, row by row, the walk takes them in 8 x 4 pixel blocks.  Every
output must be the same as without the hint, bit for bit: the samples of
both samplers (synchronous and stream-ordered), the render-only frame and
the fused sample + composite call.  The hint-free outputs are checked against
the oracle by the other parity tests; one case here also goes to the oracle
directly.  Widths cover a multiple of 32, widths that are not multiples of 8,
a width below 8, width 1, a width larger than the ray count and a partial
last row."""
import numpy as np
import pytest
import torch

from paper_2404_10272_gb300 import scenes
from _helpers import assert_same, gpu_samples, oracle_samples, slab_scene, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


def _prm(H, p, width):
    return H.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps,
                         image_width=width)


def _outputs(H, ot, dt, gv, gd, p, f, width):
    """Every output the hint reaches, as host arrays (floats as bit patterns)."""
    prm = _prm(H, p, width)
    out = {"hdda": gpu_samples(H, "hdda", ot, dt, gv, prm),
           "dense": gpu_samples(H, "dense", ot, dt, gd, prm),
           "render": to_np(H.render(ot, dt, gv, prm, f)).view(np.uint32)}
    total = int(out["hdda"][0][-1])
    n = ot.shape[0]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = H.traverse_async(ot, dt, gv, prm, H.alloc_samples(n, max(1, total)), st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    out["async"] = tuple(to_np(x) for x in (s.offsets, s.ray_idx[:total], s.t0[:total],
                                           s.t1[:total]))
    s2 = H.alloc_samples(n, max(1, total))
    rgba = H.traverse_composite(ot, dt, gv, prm, s2, f, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    out["fused"] = tuple(to_np(x) for x in (s2.offsets, s2.ray_idx[:total], s2.t0[:total],
                                           s2.t1[:total]))
    out["fused_rgba"] = to_np(rgba).view(np.uint32)
    return out


def _check(H, occ, aabbs, o, d, p, field, widths, what):
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    f = torch.from_numpy(field).cuda()
    dense_occ = torch.from_numpy(np.ascontiguousarray(occ)).cuda()
    gv, gd = H.build_vdb(dense_occ, aabbs), H.pack_dense(dense_occ, aabbs)
    base = _outputs(H, ot, dt, gv, gd, p, f, 0)
    for w in widths:
        got = _outputs(H, ot, dt, gv, gd, p, f, w)
        for k in ("hdda", "dense", "async", "fused"):
            assert_same(got[k], base[k], f"{what} width {w} {k}")
        for k in ("render", "fused_rgba"):
            assert np.array_equal(got[k], base[k]), f"{what} width {w} {k}"
    return base, ot, dt, gv


def test_unbounded_crop_in_pixel_blocks(H):
    sc = scenes.unbounded_scene()
    W, Hh = 173, 61                    # width not a multiple of 8; 10,553 rays
    o, d = scenes.unbounded_camera(W=W, H=Hh).rays()
    _check(H, sc.occ, sc.aabbs, o, d, sc.params, sc.field, [W, 1, 5, 10 ** 6], "unbounded")
    # a partial last row: the first 9,999 rays of the same image
    k = 9999
    _check(H, sc.occ, sc.aabbs, np.ascontiguousarray(o[:k]), np.ascontiguousarray(d[:k]),
           sc.params, sc.field, [W], "unbounded partial row")


def test_object_image_against_oracle(H):
    sc = scenes.object_scene()
    W, Hh = 64, 50                     # width a multiple of 32
    o, d = scenes.object_cameras(n=1, W=W, H=Hh)[0].rays()
    _check(H, sc.occ, sc.aabbs, o, d, sc.params, sc.field, [W, 40], "object")
    # and directly against the oracle with the hint on
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    gv = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    ref = oracle_samples(o, d, sc.occ, sc.aabbs, sc.params)
    assert_same(gpu_samples(H, "hdda", ot, dt, gv, _prm(H, sc.params, W)), ref,
                "object width 64 vs oracle")


def test_many_runs_in_pixel_blocks(H):
    # rays that cross more than 16 runs take the walk's later rounds
    occ, aabbs, o, d, field, p = slab_scene(64, 2, 1000, 7)
    _check(H, occ, aabbs, o, d, p, field, [40, 33], "slabs")


def test_negative_width_is_refused(H):
    sc = scenes.tiny_scene()
    o, d = scenes.tiny_camera().rays()
    gv = H.build_vdb(torch.from_numpy(sc.occ).cuda(), sc.aabbs)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    with pytest.raises(H.HddaError) as e:
        H.traverse_hdda(ot, dt, gv, _prm(H, sc.params, -1))
    assert e.value.code == H.ERR_INVALID_ARG
