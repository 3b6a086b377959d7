"""Autotuners for the z-segment length of the tile work items (node planes per CTA): ``tune`` for
the batched persistent CG solver (one choice per problem-size bucket, timed on short batched
solves) and ``tune_apply`` for the single operator apply of one mesh (timed applies).

The choice changes only how work is split among CTAs, never the arithmetic (the tile kernel's
per-node summation order does not depend on it), so results stay bitwise identical.  Choices are
cached in a JSON file keyed by GPU name, SM count and bucket.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import mf

BUCKETS = ((0, 16), (17, 32), (33, 64), (65, 1 << 30))
CANDIDATES = (4, 8, 16, 32, 64)


def _bucket(n: int) -> int:
    for i, (lo, hi) in enumerate(BUCKETS):
        if lo <= n <= hi:
            return i
    return len(BUCKETS) - 1


def cache_path() -> str:
    base = os.environ.get("MF_AUTOTUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "mf_gb300", "autotune.json")


def _device_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}"


def _load() -> dict:
    """The cache as a dict; a missing, unreadable or malformed file reads as empty."""
    try:
        with open(cache_path()) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return {}
    return d if isinstance(d, dict) else {}


def _store(d: dict) -> None:
    """Replace the cache file atomically.  Each process writes its own temporary file, so processes
    that tune at once (one per GPU) never interleave their writes; the last replacement wins."""
    path = cache_path()
    tmp = f"{path}.{os.getpid()}.tmp"
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _cached(cache: dict, key: str, candidates) -> int | None:
    """The cached choice under `key` if it is one of `candidates`, else None (the entry is tuned again)."""
    v = cache.get(key)
    if isinstance(v, int) and not isinstance(v, bool) and v in candidates:
        return v
    return None


def _time_batch(meshes, bs, xs, iters: int, reps: int = 2) -> float:
    o = mf.mf_solve_opts_default()
    o.max_iter = iters
    o.rtol = 1e-30  # run exactly `iters` iterations
    batch = mf.mf_batch_create(meshes, o)
    try:
        mf.mf_batch_solve(batch, bs, xs)
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mf.mf_batch_solve(batch, bs, xs)
            best = min(best, time.perf_counter() - t0)
        return best
    finally:
        mf.mf_batch_destroy(batch)


def tune(meshes, dims, bs, xs, iters: int = 20, use_cache: bool = True) -> dict:
    """Choose a segment length per size bucket (coordinate descent over buckets), apply it to the
    meshes with mf_set_tile_segment and return {bucket: seg}.  ``dims`` are the per-mesh node counts
    along z (the axis the tiles march along)."""
    key = _device_key()
    cache = _load() if use_cache else {}
    buckets = sorted({_bucket(d) for d in dims})
    choice = {b: 16 for b in buckets}
    cached = {b: _cached(cache, f"{key}|bucket{b}", CANDIDATES) for b in buckets}
    if use_cache and all(v is not None for v in cached.values()):
        choice = {b: int(v) for b, v in cached.items()}
    else:
        def apply_choice(ch):
            for m, d in zip(meshes, dims):
                mf.mf_set_tile_segment(m, ch[_bucket(d)])
        for b in buckets:
            best_t, best_s = float("inf"), choice[b]
            for s in CANDIDATES:
                trial = dict(choice)
                trial[b] = s
                apply_choice(trial)
                t = _time_batch(meshes, bs, xs, iters)
                if t < best_t:
                    best_t, best_s = t, s
            choice[b] = best_s
        if use_cache:
            for b in buckets:
                cache[f"{key}|bucket{b}"] = choice[b]
            _store(cache)
    for m, d in zip(meshes, dims):
        mf.mf_set_tile_segment(m, choice[_bucket(d)])
    return choice


APPLY_CANDIDATES = (0, 8, 12, 16, 20, 24, 32, 48, 64, 96, 128)


def tune_apply(mesh, reps: int = 20, use_cache: bool = True) -> int:
    """Time ``mesh.apply`` for each segment length in APPLY_CANDIDATES (0 = the library's wave-model
    default) on a random vector, keep the fastest with mf_set_tile_segment and return it.  Cached per
    GPU, physics and mesh dimensions.  The choice never changes the result bits."""
    key = f"{_device_key()}|apply|{mesh.physics}|{mesh.dims}"
    cache = _load() if use_cache else {}
    seg = _cached(cache, key, APPLY_CANDIDATES) if use_cache else None
    if seg is not None:
        mf.mf_set_tile_segment(mesh, seg)
        return seg
    n = mesh.info["n_dof"]
    x = torch.rand(n, dtype=torch.float64, device=mesh.device)
    y = torch.empty_like(x)
    best_t, best_s = float("inf"), 0
    for s in APPLY_CANDIDATES:
        if s > 0 and s > mesh.dims[2] + 1:
            continue
        mf.mf_set_tile_segment(mesh, s)
        for _ in range(3):
            mesh.apply(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            mesh.apply(x, y)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        if t < best_t:
            best_t, best_s = t, s
    mf.mf_set_tile_segment(mesh, best_s)
    if use_cache:
        cache[key] = best_s
        _store(cache)
    return best_s
