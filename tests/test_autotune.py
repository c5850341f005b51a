"""Host logic of the batch autotuner and the batch workload generator (no GPU)."""
import numpy as np
import pytest

from paper_2404_10272_gb300 import autotune, scenes


def test_choose_takes_smallest_median_and_first_on_ties():
    t = {(256, 64, 4, 0): [3.0, 1.0, 2.0], (128, 32, 2, 0): [2.0, 2.0, 2.0],
         (512, 128, 8, 0): [5, 5, 5]}
    assert autotune.choose(t) == (256, 64, 4, 0)   # medians 2.0 vs 2.0: the first timed wins
    t[(256, 64, 4, 0)] = [2.5, 2.5, 2.5]
    assert autotune.choose(t) == (128, 32, 2, 0)
    with pytest.raises(ValueError):
        autotune.choose({})


def test_tune_uses_timer_then_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("HDDA_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    calls = []

    def fake_timer(make_batch, cfg, reps, warmup):
        calls.append(cfg)
        wb, rpf, ew, wv = cfg
        return [abs(wb - 256) + abs(rpf - 64) + abs(ew - 4) + 1.0 - 0.5 * wv] * reps

    best, timings = autotune.tune(None, "wl", timer=fake_timer, device_name="dev")
    # the launch shape first, then the control flow at that shape
    assert best == (256, 64, 4, autotune.WALK_SKIP)
    assert len(calls) == len(autotune.SPACE) + 1 == 28
    assert set(timings) == set(autotune.SPACE) | {(256, 64, 4, autotune.WALK_SKIP)}

    def failing_timer(*a):
        raise AssertionError("the cache should have answered")

    best2, timings2 = autotune.tune(None, "wl", timer=failing_timer, device_name="dev")
    assert best2 == best and timings2 == timings
    # another device or workload is tuned afresh
    best3, _ = autotune.tune(None, "wl", timer=fake_timer, device_name="other")
    assert best3 == best and len(calls) == 56


def test_batch_jobs_are_seeded_and_within_bounds():
    sc1, j1 = scenes.batch_jobs(seed=7, n=6, min_side=64, max_side=96)
    sc2, j2 = scenes.batch_jobs(seed=7, n=6, min_side=64, max_side=96)
    assert [j["scene"] for j in j1] == [j["scene"] for j in j2]
    for a, b in zip(j1, j2):
        assert np.array_equal(a["rays_d"], b["rays_d"])
        assert 64 <= a["width"] <= 96 and 64 <= a["height"] <= 96
        assert a["rays_o"].shape == (a["width"] * a["height"], 3)
    for key, s in sc1.items():
        kind, levels = key
        assert s.levels == levels and 1 <= levels <= 4
        # level l's central half is the pooled finer level
        for l in range(1, levels):
            R = s.res
            q = R // 4
            pooled = s.occ[l - 1].reshape(R // 2, 2, R // 2, 2, R // 2, 2).max(axis=(1, 3, 5))
            assert np.array_equal(s.occ[l, q:q + R // 2, q:q + R // 2, q:q + R // 2] | pooled,
                                  s.occ[l, q:q + R // 2, q:q + R // 2, q:q + R // 2])


def test_signature_groups_similar_batches():
    class G:
        def __init__(self, levels, kind=1):
            self.levels, self.kind = levels, kind

    class T:
        def __init__(self, n):
            self.shape = (n, 3)

    jobs = [{"rays_o": T(1000), "grid": G(1)}, {"rays_o": T(3000), "grid": G(3)}]
    sig = autotune.signature(jobs)
    assert sig == autotune.signature(list(jobs))
    assert "jobs2" in sig and "levels[1, 3]" in sig
