"""Autotuner for the batched sampler's launch shape.

It chooses the fields of `hdda_batch_config` for a given batch by timing:
* the walk's threads per CTA;
* the rays a warp takes per work-stealing fetch;
* the 32-ray tiles per CTA of the emit;
* then, at the best of those launch shapes, the walk's control flow:
  Algorithm 1's branch form or Algorithm 2's skip form (same samples).

Every candidate builds its own plan, whose CUDA graph is captured once. It is
launched a few times untimed, then timed over `reps` launches with CUDA events.
The candidate with the smallest median wins.  Configurations are 4-tuples
(walk_block, rays_per_fetch, emit_warps, walk_variant).

Results are cached in a JSON file keyed by the device name and a signature of
the workload. The file is `$HDDA_AUTOTUNE_CACHE` if set, else `autotune.json`
in the package's build directory, so a later process reuses the choice.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Iterable

WALK_BLOCKS = (128, 256, 512)
RAYS_PER_FETCH = (32, 64, 128)
EMIT_WARPS = (2, 4, 8)
WALK_BRANCH, WALK_SKIP = 0, 1   # hdda_walk_variant
SPACE = [(wb, rpf, ew, WALK_BRANCH) for wb in WALK_BLOCKS for rpf in RAYS_PER_FETCH
         for ew in EMIT_WARPS]


def cache_path() -> str:
    env = os.environ.get("HDDA_AUTOTUNE_CACHE")
    if env:
        return env
    here = os.path.dirname(os.path.abspath(__file__))
    return os.path.join(here, "_build", "autotune.json")


def signature(jobs) -> str:
    """Workload class: job count, total rays (to a power of two), grid kind and level mix."""
    n = len(jobs)
    rays = sum(int(j["rays_o"].shape[0]) for j in jobs)
    levels = sorted({int(j["grid"].levels) for j in jobs})
    kind = {int(j["grid"].kind) for j in jobs}
    return f"jobs{n}-rays2^{max(rays, 1).bit_length()}-levels{levels}-kind{sorted(kind)}"


def load_cache(path: str | None = None) -> dict:
    try:
        with open(path or cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def store_cache(key: str, value: dict, path: str | None = None) -> None:
    path = path or cache_path()
    data = load_cache(path)
    data[key] = value
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(timings: dict) -> tuple:
    """The configuration with the smallest median time (ties: the first timed)."""
    best = None
    for cfg in timings:
        med = statistics.median(timings[cfg])
        if best is None or med < best[1]:
            best = (cfg, med)
    if best is None:
        raise ValueError("no configuration was timed")
    return best[0]


def time_config(make_batch: Callable, cfg: tuple, reps: int, warmup: int) -> list[float]:
    import torch
    b = make_batch(cfg)
    try:
        for _ in range(warmup):
            b.launch()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            b.launch()
            e1.record()
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        b.results()
        return out
    finally:
        b.free()


def tune(make_batch: Callable, key: str, space: Iterable[tuple] = SPACE, reps: int = 5,
         warmup: int = 2, timer: Callable | None = None, use_cache: bool = True,
         device_name: str | None = None) -> tuple[tuple, dict]:
    """Returns (best config, {config: [ms, ...]}).  `timer(make_batch, cfg, reps, warmup)`
    replaces the CUDA timing (tests pass a fake one)."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    full_key = f"{device_name}|{key}"
    if use_cache:
        hit = load_cache().get(full_key)
        if hit:
            return tuple(hit["config"]), {tuple(json.loads(k)): v for k, v in hit["timings"].items()}
    timer = timer or time_config
    timings = {tuple(cfg): timer(make_batch, tuple(cfg), reps, warmup) for cfg in space}
    shape = choose(timings)
    alt = shape[:3] + (WALK_SKIP if shape[3] == WALK_BRANCH else WALK_BRANCH,)
    if alt not in timings:
        timings[alt] = timer(make_batch, alt, reps, warmup)
    best = choose(timings)
    if use_cache:
        store_cache(full_key, {"config": list(best),
                               "timings": {json.dumps(list(k)): v for k, v in timings.items()}})
    return best, timings
