"""Admission and continuous batching of the render server, with a fake executor
(no GPU): FIFO order, slot and memory limits, joining while others run, re-runs."""
import threading
import time

import numpy as np

from paper_2404_10272_gb300 import serve


def _req(i, n, scene=0):
    return serve.Request(rid=i, scene=scene, rays_o=np.zeros((n, 3), np.float32),
                         rays_d=np.zeros((n, 3), np.float32))


def test_admission_fifo_budget_and_slots():
    adm = serve.Admission(budget_bytes=10_000_000, slots=2, samples_per_ray_hint=10)
    for i, n in enumerate([1000, 50_000, 1000, 1000]):
        adm.push(_req(i, n))
    first = adm.pop_admissible()
    assert [r.rid for r in first] == [0]          # request 1 does not fit next to 0
    assert adm.in_use <= adm.budget
    adm.release(first[0])
    second = adm.pop_admissible()
    assert [r.rid for r in second] == [1]         # alone it may exceed the budget
    assert adm.pop_admissible() == []             # nothing overtakes the head... (2 waits)
    adm.release(second[0])
    third = adm.pop_admissible()
    assert [r.rid for r in third] == [2, 3]       # slots = 2
    assert adm.busy == 2


def test_samples_per_ray_learned_and_resize():
    adm = serve.Admission(budget_bytes=1 << 40, slots=4, samples_per_ray_hint=64)
    r = _req(0, 1000, scene=3)
    adm.push(r)
    adm.pop_admissible()
    before = adm.in_use
    adm.resize(r, 500_000)
    assert adm.in_use - before == r.reserved - (before)
    r.samples = 20_000
    adm.release(r)
    assert adm.in_use == 0 and abs(adm.spr[3] - 20.0) < 1e-9
    # the estimate follows a heavier view at once and decays slowly after it
    r2 = _req(1, 1000, scene=3)
    r2.samples, r2.reserved = 40_000, 0
    adm.busy += 1
    adm.release(r2)
    assert abs(adm.spr[3] - 40.0) < 1e-9
    r3 = _req(2, 1000, scene=3)
    r3.samples, r3.reserved = 1_000, 0
    adm.busy += 1
    adm.release(r3)
    assert abs(adm.spr[3] - 0.97 * 40.0) < 1e-9


class FakeExec:
    def __init__(self):
        self.lock = threading.Lock()
        self.active = 0
        self.peak = 0
        self.order = []
        self.retried = set()

    def __call__(self, slot, req, reserved):
        with self.lock:
            self.active += 1
            self.peak = max(self.peak, self.active)
            self.order.append(req.rid)
        try:
            if req.rid == 3 and req.rid not in self.retried:
                self.retried.add(req.rid)
                raise serve.NeedMore(req.n_rays * 200)
            time.sleep(0.002 + req.n_rays * 1e-7)
            req.samples = req.n_rays * 5
            req.rgba = np.full((req.n_rays, 4), req.rid, np.float32)
        finally:
            with self.lock:
                self.active -= 1


def test_server_overlaps_and_completes_everything():
    ex = FakeExec()
    srv = serve.RenderServer(ex, slots=3, budget_bytes=1 << 34, samples_per_ray_hint=5)
    reqs = [_req(i, 1000 + 37 * i) for i in range(20)]
    for r in reqs[:10]:
        srv.submit(r)
    time.sleep(0.005)
    for r in reqs[10:]:             # arrive while the first ones are on the "GPU"
        srv.submit(r)
    srv.close()
    assert len(srv.completed) == 20 and all(r.error is None for r in reqs)
    assert ex.peak == 3              # slots fill up, never beyond
    assert reqs[3].retries == 1
    assert all(float(r.rgba[0, 0]) == r.rid for r in reqs)
    # admission is FIFO
    assert sorted(reqs, key=lambda r: r.admitted) == sorted(reqs, key=lambda r: r.rid)
    # later arrivals joined before the earlier batch had finished (continuous batching)
    first_done = min(r.done for r in reqs[:10])
    assert min(r.admitted for r in reqs[10:]) < max(r.done for r in reqs[:10])
    assert first_done < max(r.done for r in reqs)
    s = serve.summary(reqs, 1.0)
    assert s["requests"] == 20 and s["errors"] == 0 and s["p99_ms"] >= s["p50_ms"]


def test_failed_request_does_not_stop_the_server():
    def boom(slot, req, reserved):
        if req.rid == 1:
            raise RuntimeError("bad request")
        req.samples = 1
    srv = serve.RenderServer(boom, slots=2, budget_bytes=1 << 30)
    reqs = [_req(i, 10) for i in range(4)]
    for r in reqs:
        srv.submit(r)
    srv.close()
    assert [r.error is not None for r in reqs] == [False, True, False, False]


def test_admission_without_sample_buffers():
    """Render mode: a request costs bytes per ray only, whatever the scene's history."""
    adm = serve.Admission(budget_bytes=10_000, slots=8, bytes_per_ray=100, bytes_per_sample=0)
    reqs = [serve.Request(rid=i, scene=0, rays_o=np.zeros((30, 3)), rays_d=np.zeros((30, 3)))
            for i in range(5)]
    for r in reqs:
        adm.push(r)
    got = adm.pop_admissible()
    assert [r.rid for r in got] == [0, 1, 2]          # 3 x 3000 bytes fit in 10000
    assert all(r.reserved == 3000 for r in got)
    r = got[0]
    r.samples = 10 ** 6                               # no effect on later estimates
    adm.release(r)
    assert adm.estimate_bytes(reqs[3]) == 3000
