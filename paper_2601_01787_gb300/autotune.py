"""Autotuner of the code pass's tile shape.

The code pass (the first phase of msz_correct / msz_correct_batch) walks 3D
fields in tiles of 128 (x) by 8 (y) vertices -- fixed by the warp layout -- and
a tunable number of z-planes per tile.  Deeper tiles re-read fewer halo planes;
shallower tiles balance the tile queue better on small fields.  The tuner times
the candidates on a synthetic field of the same size class with the device
time of that phase (``stats["codes_ns"]``) and caches the winner per GPU and
size class in a JSON file.  The choice changes speed only, never results.
"""
from __future__ import annotations

import json
import math
import os
import threading

CANDIDATES = (8, 16, 32, 64)
DEFAULT = 32
_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.environ.get("MSZ_AUTOTUNE_CACHE", os.path.join(_HERE, "_build", "autotune.json"))
_lock = threading.Lock()


def size_class(shape) -> str:
    """Bucket of a (nz, ny, nx) shape: nz and the x-y plane size, each rounded to
    the nearest power of two."""
    nz, ny, nx = (int(v) for v in shape)
    bz = 1 << max(0, round(math.log2(max(nz, 1))))
    bp = 1 << max(0, round(math.log2(max(nx * ny, 1))))
    return f"z{bz}_p{bp}"


def _load() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(d: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _device_key() -> str:
    import torch
    return torch.cuda.get_device_name().replace(" ", "_")


def lookup(shape, device_key: str | None = None) -> int:
    """Cached tile depth for this size class (DEFAULT when never tuned)."""
    key = f"{device_key or _device_key()}|{size_class(shape)}"
    return int(_load().get(key, {}).get("tile_z", DEFAULT))


def record(shape, tile_z: int, timings: dict, device_key: str) -> None:
    with _lock:
        d = _load()
        d[f"{device_key}|{size_class(shape)}"] = {"tile_z": int(tile_z),
                                                  "codes_ms": {str(k): v for k, v in timings.items()}}
        _save(d)


def tune(shape, reps: int = 3, seed: int = 77) -> int:
    """Time every candidate on a synthetic field of `shape` and cache the best."""
    import torch

    from . import api, synth
    fl = synth.perlin3d_prequant(tuple(shape), seed=seed, eb_rel=1e-4)
    f = torch.from_numpy(fl.f).cuda()
    fh = torch.from_numpy(fl.fhat).cuda()
    timings = {}
    for tz in CANDIDATES:
        best = None
        for _ in range(reps + 1):
            r = api.correct(f, fh, fl.xi, max_sweeps=1, edit_capacity=0, tile_z=tz)
            t = r.stats["codes_ns"] / 1e6
            best = t if best is None else min(best, t)
        timings[tz] = round(best, 5)
    winner = min(timings, key=timings.get)
    record(shape, winner, timings, _device_key())
    return winner


def tile_z_for(shapes, tune_missing: bool = False) -> list[int]:
    """Tile depth for each shape: the cached choice of its size class, tuning the
    classes never seen when asked to."""
    out = []
    seen = {}
    dk = _device_key()
    cache = _load()
    for s in shapes:
        c = size_class(s)
        if c not in seen:
            hit = cache.get(f"{dk}|{c}")
            seen[c] = int(hit["tile_z"]) if hit else (tune(s) if tune_missing else DEFAULT)
        out.append(seen[c])
    return out
