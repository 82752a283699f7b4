"""Autotuner of the batched form: picks the hdiff tile, the K-blocking (levels
per hdiff work item) and the vadv block width for a given ensemble, and
caches the choice.

The cache is keyed by a fingerprint of what the choice depends on: the
members' domains, the dtype, the precision mode, the GPU and the library
version, so re-running with the same ensemble shapes reuses the plan
parameters without timing again (cf. GT4Py's fingerprint cache of generated
stencils, Sec. 2.3).
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

import torch

from . import gtb

VADV_WARPS = (1, 2, 4)
HDIFF_TILES = (0, 1)
HDIFF_LEVELS = (4, 8, 16, 0)


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "gtb", "autotune.json")


def fingerprint(members, prec: str) -> str:
    dt = str(members[0]["in"].data.dtype)
    shapes = sorted(tuple(int(x) for x in m["domain"]) for m in members)
    key = {"shapes": shapes, "dtype": dt, "prec": prec, "gpu": torch.cuda.get_device_name(),
           "lib": gtb.version()}
    return hashlib.sha256(json.dumps(key, sort_keys=True).encode()).hexdigest()[:24]


def time_plan(members, config, *, prec, dtr_stage=3.0 / 20.0, beta_v=0.0, reps=5) -> float:
    """Median milliseconds of one graph replay."""
    plan = gtb.BatchPlan(members, dtr_stage=dtr_stage, beta_v=beta_v, prec=prec, config=config)
    try:
        plan.run()
        plan.run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.run()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        gtb.device_status()
        return statistics.median(ts)
    finally:
        plan.close()


def tune(members, *, prec="native", dtr_stage=3.0 / 20.0, beta_v=0.0, cache_path=None, reps=5, force=False):
    """Best config for this ensemble: from the cache, or by a coordinate search
    (vadv block width, then hdiff tile x K-blocking).  Returns (config, log)."""
    cache_path = cache_path or default_cache_path()
    fp = fingerprint(members, prec)
    cache = {}
    if os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    if fp in cache and not force:
        return cache[fp]["config"], {"cached": True, "fingerprint": fp}
    log = []
    best = dict(gtb.DEFAULT_BATCH_CONFIG)
    best_t = None
    for vw in VADV_WARPS:
        cfg = dict(best, vadv_warps=vw)
        t = time_plan(members, cfg, prec=prec, dtr_stage=dtr_stage, beta_v=beta_v, reps=reps)
        log.append((cfg, t))
        if best_t is None or t < best_t:
            best, best_t = cfg, t
    for tile in HDIFF_TILES:
        for lv in HDIFF_LEVELS:
            cfg = dict(best, hdiff_tile=tile, hdiff_levels=lv)
            if cfg == best:
                continue
            t = time_plan(members, cfg, prec=prec, dtr_stage=dtr_stage, beta_v=beta_v, reps=reps)
            log.append((cfg, t))
            if t < best_t:
                best, best_t = cfg, t
    cache[fp] = {"config": best, "ms": best_t}
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return best, {"cached": False, "fingerprint": fp, "best_ms": best_t, "tried": log}
