"""Batched sampling: one plan over many jobs gives, job by job, exactly the samples of
the single-call sampler, with the graph or without, for any launch configuration and
across repeated launches; capacity is checked per job."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_10272_gb300 import scenes
from _helpers import assert_same, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    return hdda


@pytest.fixture(scope="module")
def workload(H):
    sc, jobs = scenes.batch_jobs(seed=7, n=10, min_side=40, max_side=120)
    grids = {k: H.build_vdb(torch.from_numpy(s.occ).cuda(), s.aabbs) for k, s in sc.items()}
    dense = {k: H.pack_dense(torch.from_numpy(s.occ).cuda(), s.aabbs) for k, s in sc.items()}
    specs = []
    for j in jobs:
        s = sc[j["scene"]]
        p = s.params
        specs.append(dict(rays_o=torch.from_numpy(j["rays_o"]).cuda(),
                          rays_d=torch.from_numpy(j["rays_d"]).cuda(), key=j["scene"],
                          params=H.make_params(p.near, p.far, p.step, p.cone, p.max_step,
                                               p.max_steps)))
    # a job without rays
    specs.append(dict(rays_o=torch.zeros((0, 3), device="cuda"), rays_d=torch.zeros((0, 3), device="cuda"),
                      key=specs[0]["key"], params=specs[0]["params"]))
    return sc, grids, dense, specs


def _jobs(H, specs, grids, fn, slack=0):
    jobs, refs = [], []
    for sp in specs:
        g = grids[sp["key"]]
        ref = fn(sp["rays_o"], sp["rays_d"], g, sp["params"])
        refs.append(tuple(to_np(x) for x in ref.trimmed()))
        out = H.alloc_samples(sp["rays_o"].shape[0], max(1, ref.total + slack))
        jobs.append(dict(rays_o=sp["rays_o"], rays_d=sp["rays_d"], grid=g, params=sp["params"],
                         out=out))
    return jobs, refs


@pytest.mark.parametrize("config,graph", [((256, 64, 4), True), ((128, 32, 2), False),
                                          ((512, 128, 8), True), ((256, 64, 4, 1), True),
                                          ((128, 32, 8, 1), False)])
def test_batch_matches_single_calls(H, workload, config, graph):
    sc, grids, _, specs = workload
    jobs, refs = _jobs(H, specs, grids, H.traverse_hdda, slack=5)
    b = H.Batch(jobs, config=config, use_graph=graph)
    for rep in range(2):   # a replay gives the same samples again
        for jb in jobs:
            jb["out"].offsets.fill_(-1)
            jb["out"].t0.fill_(-1.0)
        b.launch()
        totals, status = b.results()
        assert status == [0] * len(jobs)
        for i, (jb, ref) in enumerate(zip(jobs, refs)):
            assert totals[i] == ref[0][-1]
            assert_same(tuple(to_np(x) for x in jb["out"].trimmed()), ref, f"job {i} rep {rep}")
    b.free()


def test_dense_batch_and_oracle(H, workload):
    sc, _, dense, specs = workload
    jobs, refs = _jobs(H, specs[:4], dense, H.traverse_dense)
    b = H.Batch(jobs)
    b.launch()
    b.results()
    for i, (sp, jb) in enumerate(zip(specs[:4], jobs)):
        s = sc[sp["key"]]
        p = s.params
        o, d = to_np(sp["rays_o"]), to_np(sp["rays_d"])
        sel = np.arange(0, o.shape[0], 7)
        ref = oracle.sample(o[sel], d[sel], s.occ, s.aabbs, p.near, p.far, p.step, p.cone,
                            p.max_step, p.max_steps)
        off, idx, t0, t1 = (to_np(x) for x in jb["out"].trimmed())
        for k, r in enumerate(sel):
            assert np.array_equal(t0[off[r]:off[r + 1]].view(np.uint32),
                                  ref[2][ref[0][k]:ref[0][k + 1]].view(np.uint32))
    b.free()


def test_capacity_is_per_job(H, workload):
    sc, grids, _, specs = workload
    jobs, refs = _jobs(H, specs[:3], grids, H.traverse_hdda)
    small = H.alloc_samples(specs[1]["rays_o"].shape[0], max(1, refs[1][0][-1] // 2))
    jobs[1]["out"] = small
    b = H.Batch(jobs)
    b.launch()
    totals, status = b.results(check=False)
    assert status == [0, H.ERR_CAPACITY, 0]
    assert totals[1] == refs[1][0][-1]
    with pytest.raises(H.HddaError):
        b.results()
    for i in (0, 2):
        assert_same(tuple(to_np(x) for x in jobs[i]["out"].trimmed()), refs[i], f"job {i}")
    b.free()


def test_mixed_kinds_rejected(H, workload):
    sc, grids, dense, specs = workload
    jobs, _ = _jobs(H, specs[:2], grids, H.traverse_hdda)
    jobs[1]["grid"] = dense[specs[1]["key"]]
    with pytest.raises(H.HddaError):
        H.Batch(jobs)
