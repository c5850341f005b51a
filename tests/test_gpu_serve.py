"""Render server on the GPU: a frame is the same alone and in a mix of concurrent
requests (the compositor's tolerance is 1e-5; the kernels are deterministic, so the
frames agree exactly), and equal to the direct API calls."""
import numpy as np
import pytest
import torch

from paper_2404_10272_gb300 import scenes, serve

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    sc = [scenes.tiny_scene(), scenes.object_scene()]
    ex = serve.GpuExecutor(sc, slots=4)
    ex.warm()
    return hdda, sc, ex


def _rays(seed, W, H):
    cam = scenes.orbit_camera(np.random.default_rng(seed), 4.0, W, H, 0.69)
    o, d = cam.rays()
    return torch.from_numpy(o).pin_memory(), torch.from_numpy(d).pin_memory()


def test_alone_equals_mixed_and_direct(setup):
    hdda, sc, ex = setup
    o, d = _rays(1, 320, 240)
    alone = serve.Request(rid=0, scene=1, rays_o=o, rays_d=d, width=320)
    srv = serve.RenderServer(ex, slots=4, budget_bytes=4 << 30)
    srv.submit(alone)
    srv.close()
    assert alone.error is None
    srv = serve.RenderServer(ex, slots=4, budget_bytes=4 << 30, samples_per_ray_hint=2)
    mix = []
    for i in range(12):
        oo, dd = _rays(100 + i, 64 + 40 * i, 48 + 30 * i)
        mix.append(serve.Request(rid=i + 1, scene=i % 2, rays_o=oo, rays_d=dd,
                                 width=64 + 40 * i))
    target = serve.Request(rid=99, scene=1, rays_o=o, rays_d=d, width=320)
    for r in mix[:6] + [target] + mix[6:]:
        srv.submit(r)
    srv.close()
    assert all(r.error is None for r in mix + [target])
    assert srv.max_concurrent > 1
    assert target.samples == alone.samples
    diff = (target.rgba - alone.rgba).abs().max().item()
    assert diff <= TOL
    # the low hint forces re-runs at the exact size somewhere in the mix
    assert sum(r.retries for r in mix + [target]) > 0
    # direct API, with the rays in index order (the server passed the image width)
    p = sc[1].params
    prm = hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    s = hdda.traverse_hdda(o.cuda(), d.cuda(), ex.grids[1], prm)
    rgba = hdda.composite(o.cuda(), d.cuda(), s, ex.fields[1]).cpu()
    assert s.total == alone.samples
    assert (rgba - alone.rgba).abs().max().item() <= TOL


def test_render_mode_alone_equals_mixed_and_direct(setup):
    hdda, sc, _ = setup
    ex = serve.GpuExecutor(sc, slots=4, mode="render")
    ex.warm()
    o, d = _rays(2, 320, 240)
    alone = serve.Request(rid=0, scene=1, rays_o=o, rays_d=d, width=320)
    srv = serve.RenderServer(ex, slots=4, budget_bytes=1 << 30)
    srv.submit(alone)
    srv.close()
    assert alone.error is None and alone.retries == 0
    srv = serve.RenderServer(ex, slots=4, budget_bytes=1 << 30)
    mix = []
    for i in range(12):
        oo, dd = _rays(200 + i, 64 + 40 * i, 48 + 30 * i)
        mix.append(serve.Request(rid=i + 1, scene=i % 2, rays_o=oo, rays_d=dd,
                                 width=64 + 40 * i))
    target = serve.Request(rid=99, scene=1, rays_o=o, rays_d=d, width=320)
    for r in mix[:6] + [target] + mix[6:]:
        srv.submit(r)
    srv.close()
    assert all(r.error is None and r.retries == 0 for r in mix + [target])
    assert srv.max_concurrent > 1
    assert torch.equal(target.rgba, alone.rgba)
    # direct API with the rays in index order (bit for bit: the server passed the image
    # width), and the sample-buffer path within the compositor's tolerance
    p = sc[1].params
    prm = hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    direct = hdda.render(o.cuda(), d.cuda(), ex.grids[1], prm, ex.fields[1]).cpu()
    assert torch.equal(direct, alone.rgba)
    s = hdda.traverse_hdda(o.cuda(), d.cuda(), ex.grids[1], prm)
    two = hdda.composite(o.cuda(), d.cuda(), s, ex.fields[1]).cpu()
    assert (two - alone.rgba).abs().max().item() <= 2 * TOL


def test_batched_mode_alone_equals_mixed_and_direct(setup):
    # "batched": a slot samples every ready request of a tick in one hdda_batch launch
    # (work stealing across requests and scenes), then composites each frame.  A frame
    # is the same alone, batched with others, and through the direct API; frames that
    # outgrow their reservation re-run alone at the exact size.
    hdda, sc, _ = setup
    ex = serve.GpuExecutor(sc, slots=2, mode="batched")
    ex.warm()
    o, d = _rays(3, 320, 240)
    alone = serve.Request(rid=0, scene=1, rays_o=o, rays_d=d)
    srv = serve.RenderServer(ex, slots=2, budget_bytes=4 << 30)
    srv.submit(alone)
    srv.close()
    assert alone.error is None
    srv = serve.RenderServer(ex, slots=2, budget_bytes=4 << 30, samples_per_ray_hint=2,
                             max_batch=8)
    mix = []
    for i in range(14):
        oo, dd = _rays(300 + i, 64 + 40 * i, 48 + 30 * i)
        mix.append(serve.Request(rid=i + 1, scene=i % 2, rays_o=oo, rays_d=dd))
    target = serve.Request(rid=99, scene=1, rays_o=o, rays_d=d)
    for r in mix[:7] + [target] + mix[7:]:
        srv.submit(r)
    srv.close()
    assert all(r.error is None for r in mix + [target])
    assert target.samples == alone.samples
    assert torch.equal(target.rgba, alone.rgba)
    # the low hint makes some frames outgrow their reservation: they re-ran alone
    assert sum(r.retries for r in mix + [target]) > 0
    p = sc[1].params
    prm = hdda.make_params(p.near, p.far, p.step, p.cone, p.max_step, p.max_steps)
    s = hdda.traverse_hdda(o.cuda(), d.cuda(), ex.grids[1], prm)
    direct = hdda.composite(o.cuda(), d.cuda(), s, ex.fields[1]).cpu()
    assert s.total == alone.samples
    assert torch.equal(direct, alone.rgba)
