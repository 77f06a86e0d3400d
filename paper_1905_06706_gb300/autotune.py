"""Closed-loop autotuner of the sampler's free knobs (client side).

The sample is exact whatever the deepest quadtree level (the level cap, a field of every
request): it only moves work between the all-pairs tests of neighbouring cells and the
geometric jumps over distant ones.  The library's default cap comes from a cost balance
(about 2^(d/2) vertices per cell at T > 0); this module times the default and its
neighbours on a sample request of each request class on the GPU at hand and keeps the
fastest, and times the server's worker count on a closed-loop sample of a request mix.
The results go to a JSON file and are applied by setting ``level_cap`` in the requests,
so every graph stays a deterministic function of its parameters (a tuned cap draws a
different, equally exact graph than the default cap).

Classes: dimension d, T = 0 or T > 0, and n in [10^3, 10^4), [10^4, 10^5), [10^5, oo).
"""
from __future__ import annotations

import json
import math
import statistics
import time

N_BUCKETS = (10_000, 100_000)  # upper bounds of the first two n classes


def default_level_cap(n: int, d: int, T: float) -> int:
    """The library's default deepest level (same rule as its C code)."""
    bl = int(n).bit_length()
    a = 32 // d
    b = (2 * bl - 2 - d) // (2 * d) if T > 0.0 else (bl + 4) // d
    return max(1, min(a, b))


def request_class(n: int, d: int, T: float) -> str:
    nb = 0 if n < N_BUCKETS[0] else (1 if n < N_BUCKETS[1] else 2)
    return f"d{d}_{'T0' if T == 0.0 else 'T>0'}_n{nb}"


def _time_calls(gg, torch, fn, steps: int, warmup: int) -> float:
    for _ in range(warmup):
        fn()
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if r.status != gg.GIRG_OK:
            raise RuntimeError(gg.status_string(r.status))
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def tune_level_caps(samples: dict, offsets=(-1, 0, 1), steps: int = 3, warmup: int = 1) -> dict:
    """samples: {class name: request parameters (n, d, beta, T, avg_deg, seed)}.  For each
    class, times count-only generation at the default cap plus each offset and returns
    {class: {"level_cap": best, "default": default, "ms": {cap: median ms}}}."""
    import torch

    import paper_1905_06706_gb300 as gg
    out = {}
    for name, q in samples.items():
        base = default_level_cap(q["n"], q["d"], q["T"])
        caps = sorted({min(32 // q["d"], max(1, base + o)) for o in offsets})
        times = {}
        for lc in caps:
            times[lc] = _time_calls(gg, torch,
                                    lambda: gg.girg_generate(None, level_cap=lc, **q),
                                    steps, warmup)
        best = min(times, key=times.get)
        out[name] = {"level_cap": best, "default": base,
                     "ms": {str(k): v for k, v in times.items()}}
    return out


def class_samples(requests) -> dict:
    """One representative request per class of a request list: the one with the median n."""
    by = {}
    for q in requests:
        by.setdefault(request_class(q["n"], q["d"], q["T"]), []).append(q)
    out = {}
    for name, qs in by.items():
        qs = sorted(qs, key=lambda q: q["n"])
        out[name] = dict(qs[len(qs) // 2])
    return out


def tune_workers(run_mix, grid=(4, 8, 16)) -> dict:
    """run_mix(workers) -> edges/s of a closed-loop sample; returns the best and all."""
    rates = {w: run_mix(w) for w in grid}
    return {"workers": max(rates, key=rates.get), "edges_per_s": rates}


def apply(table: dict, q: dict) -> dict:
    """The request with the tuned level cap of its class (unchanged if the class was not
    tuned or the caller fixed a cap)."""
    if q.get("level_cap"):
        return q
    ent = table.get("level_cap", {}).get(request_class(q["n"], q["d"], q["T"]))
    return dict(q, level_cap=ent["level_cap"]) if ent else q


def save(table: dict, path: str) -> None:
    import torch
    table = dict(table, device=torch.cuda.get_device_name(), time=time.time())
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


def expected_gain(table: dict) -> float:
    """Geometric mean over the classes of default time / tuned time."""
    r = [ent["ms"][str(ent["default"])] / ent["ms"][str(ent["level_cap"])]
         for ent in table.get("level_cap", {}).values() if str(ent["default"]) in ent["ms"]]
    return math.exp(sum(math.log(x) for x in r) / len(r)) if r else 1.0
