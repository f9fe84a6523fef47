"""Autotuner for the layout and launch shape of the solves.

For a single system it times the solve over the slice heights (rows per
sliced-ELL slice: 32, 64, 128); for a batch it also tries team schedules
(largest team, work-per-block scale).  Each candidate is timed with CUDA
events on the calling stream after one warm-up solve, best of `repeats`,
with the L2 flushed before every timed solve (as the benchmark does).
Results are cached in a JSON file keyed by the problem's shape, so a later
run with the same sizes reuses the choice without timing.

All solves go through the library's C ABI; this module only chooses
parameters.
"""
import hashlib
import json
import os

import numpy as np
import torch

from . import ldupcg

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "cache.json")

SLICE_ROWS = (32, 64, 128)
SCHEDULES = ((32, 1.0), (16, 0.5), (8, 2.0), (1, 1.0))


def _key(kind, sizes, faces, extra):
    h = hashlib.sha256()
    h.update(np.asarray(sizes, dtype=np.int64).tobytes())
    h.update(np.asarray(faces, dtype=np.int64).tobytes())
    h.update(json.dumps(extra, sort_keys=True).encode())
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{kind}:{dev}:{h.hexdigest()[:24]}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    data = _load()
    data[key] = value
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


_FLUSH = None


def _flush_l2():
    """Overwrite a buffer twice the size of the 129 MB L2, as the benchmark
    does before every timed solve, so that candidates are ranked under the
    conditions they are measured in."""
    global _FLUSH
    if _FLUSH is None:
        _FLUSH = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    _FLUSH.fill_(1.0)


def _time(call, repeats):
    call()                                   # warm-up
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        _flush_l2()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return best


# (replacement period, tau) pairs tried for the mixed solve.  The float
# iteration count is sensitive to where the replacements fall: at 128^3
# (lognormal diffusivity) only period 16 with the tau test reaches the FP64
# method's 752 iterations, while at 96^3 every 24 or 32 iterations keeps its
# 616 with half the replacements.
RR_RULES = ((16, 0.3), (16, 0.2), (14, 0.0), (12, 0.0), (20, 0.3), (24, 0.0), (32, 0.0))


def tune_single(system, precision="mixed", tol=1e-8, repeats=3, use_cache=True,
                slice_rows=SLICE_ROWS, **solve_kw):
    """Best slice height (and, for the mixed solve, replacement period and
    tau) for pcg_solve ('pcg') / pipecg_solve ('fp64', 'mixed') on this
    system."""
    rules = (RR_RULES if precision == "mixed" and "rr_period" not in solve_kw
             and "tau" not in solve_kw else (None,))
    key = _key("single", [system.n], [system.nfaces],
               dict(precision=precision, tol=tol, slice_rows=list(slice_rows),
                    rules=[list(r) for r in rules if r is not None], **solve_kw))
    if use_cache:
        hit = _load().get(key)
        if hit:
            return hit
    b = torch.as_tensor(system.b, device="cuda")
    x = torch.zeros_like(b)
    results = []
    for C in slice_rows:
        A = ldupcg.from_system(system, slice_rows=C)
        for rule in rules:
            kw = dict(solve_kw)
            if rule is not None:
                kw["rr_period"], kw["tau"] = rule

            def call():
                x.zero_()
                if precision == "pcg":
                    ldupcg.pcg_solve(A, b, x, tol=tol)
                else:
                    ldupcg.pipecg_solve(A, b, x, tol=tol, precision=precision, **kw)

            res = {"slice_rows": C, "seconds": _time(call, repeats)}
            if rule is not None:
                res["rr_period"], res["tau"] = rule
            results.append(res)
        A.close()
    best = min(results, key=lambda r: r["seconds"])
    best = dict(best, candidates=results)
    _store(key, best)
    return best


def tune_batched(systems, precision="mixed", tol=1e-8, repeats=3, use_cache=True, **solve_kw):
    """Best (slice height, team schedule) for pcg_solve_batched on this batch."""
    sizes = [s.n for s in systems]
    faces = [s.nfaces for s in systems]
    key = _key("batched", sizes, faces, dict(precision=precision, tol=tol, **solve_kw))
    if use_cache:
        hit = _load().get(key)
        if hit:
            return hit
    b = torch.as_tensor(np.concatenate([s.b for s in systems]), device="cuda")
    x = torch.zeros_like(b)
    results = []
    for C in SLICE_ROWS:
        A = ldupcg.from_systems(systems, slice_rows=C)
        for max_team, scale in SCHEDULES:
            ldupcg.ldu_batch_schedule(A, max_team=max_team, team_work_scale=scale)

            def call():
                x.zero_()
                ldupcg.pcg_solve_batched(A, b, x, tol=tol, precision=precision, **solve_kw)

            results.append({"slice_rows": C, "max_team": max_team, "team_work_scale": scale,
                            "seconds": _time(call, repeats)})
        A.close()
    best = min(results, key=lambda r: r["seconds"])
    best = dict(best, candidates=results)
    _store(key, best)
    return best
