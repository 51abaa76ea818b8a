"""Autotuner of libgap's schedule options.

The kernels' tile shapes are fixed at compile time.  What varies with the problem is
the schedule around them:
- how many fits of a batch run at once: gap_fit_batched's "batch_lanes" worker
  contexts, each with its own stream;
- how much work the FP32 QR does per panel and per trailing update ("cqr_passes",
  "qr_passes"), against the FP64 refinement iterations that work saves.  A rougher QR
  is cheaper, but it is a rougher preconditioner.

The tuner times each candidate on the caller's own problem: device time, CUDA events
on the context's stream, with every candidate run once untimed first so that
workspace growth is not timed.  It keeps the fastest candidate whose fit converged,
applies it to the context, and records it in a JSON cache.  The cache is keyed by the
GPU, the precision and a shape class (powers of two of the design rows and of M, and
d), so later problems of the same class skip the timing.
"""
import json
import math
import os
from typing import Callable, Optional, Sequence

FIT_CANDIDATES = ({"qr_passes": 1, "cqr_passes": 1}, {"qr_passes": 1, "cqr_passes": 2},
                  {"qr_passes": 3, "cqr_passes": 2})
BATCH_CANDIDATES = ({"batch_lanes": 2}, {"batch_lanes": 4}, {"batch_lanes": 8})


def _bucket(x: int) -> int:
    return int(round(math.log2(max(1, int(x)))))


def fit_key(device: str, precision: str, rows: int, M: int, d: int) -> str:
    return "%s|%s|fit|rows~2^%d|M~2^%d|d%d" % (device, precision, _bucket(rows), _bucket(M), d)


def batch_key(device: str, precision: str, rows: Sequence[int], Ms: Sequence[int]) -> str:
    return "%s|%s|batch|n%d|rows~2^%d|M~2^%d" % (device, precision, len(rows), _bucket(sum(rows)),
                                                 _bucket(max(Ms) if Ms else 1))


class TuneCache:
    """Best options per key, kept in a JSON file (or in memory when path is None)."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get(self, key: str) -> Optional[dict]:
        e = self.entries.get(key)
        return dict(e["options"]) if e else None

    def put(self, key: str, options: dict, ms: float, trials: list):
        self.entries[key] = {"options": dict(options), "ms": ms, "trials": trials}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def choose(candidates: Sequence[dict], run: Callable[[dict], Optional[float]]):
    """Run every candidate; return (options, ms, trials) of the fastest one that
    succeeded (run returns its time in ms, or None when the candidate failed)."""
    trials = []
    for opts in candidates:
        trials.append({"options": dict(opts), "ms": run(dict(opts))})
    ok = [(t["ms"], i) for i, t in enumerate(trials) if t["ms"] is not None]
    if not ok:
        raise RuntimeError("no candidate schedule ran: %s" % trials)
    ms, i = min(ok)
    return dict(trials[i]["options"]), ms, trials


def _timed(ctx, fn):
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(ctx.stream)
    out = fn()
    ev1.record(ctx.stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), out


def _apply(ctx, opts: dict):
    for k, v in opts.items():
        ctx.set_option(k, v)


def tune_fit(ctx, problem, c_out, cache: Optional[TuneCache] = None, candidates=FIT_CANDIDATES) -> dict:
    """Pick the FP32 QR's passes for fits shaped like `problem` on ctx (mixed precisions;
    FP64 has nothing to tune).  Leaves the chosen options set on ctx."""
    import torch
    from . import design_rows
    if ctx.precision == "fp64":
        return {}
    s = problem.struct
    key = fit_key(torch.cuda.get_device_name(), ctx.precision, design_rows(problem), s.n_sparse, s.d)
    hit = cache.get(key) if cache else None
    if hit is not None:
        _apply(ctx, hit)
        return hit

    def fit():
        ctx.assemble(problem)
        ctx.factor()
        return ctx.solve(c_out, check=False)

    def run(opts):
        _apply(ctx, opts)
        fit()
        ms, info = _timed(ctx, fit)
        return ms if info["converged"] else None

    best, ms, trials = choose(candidates, run)
    _apply(ctx, best)
    if cache is not None:
        cache.put(key, best, ms, trials)
    return best


def tune_batched(ctx, problems, c_outs, cache: Optional[TuneCache] = None, candidates=BATCH_CANDIDATES) -> dict:
    """Pick the fits in flight of gap_fit_batched for this batch on ctx.  Leaves the
    chosen options set on ctx."""
    import torch
    from . import GapError, design_rows
    rows = [design_rows(p) for p in problems]
    Ms = [p.struct.n_sparse for p in problems]
    key = batch_key(torch.cuda.get_device_name(), ctx.precision, rows, Ms)
    hit = cache.get(key) if cache else None
    if hit is not None:
        _apply(ctx, hit)
        return hit

    def run(opts):
        _apply(ctx, opts)
        try:
            ctx.fit_batched(problems, c_outs)
            ms, infos = _timed(ctx, lambda: ctx.fit_batched(problems, c_outs))
        except GapError:
            return None
        return ms if all(i["converged"] for i in infos) else None

    best, ms, trials = choose(candidates, run)
    _apply(ctx, best)
    if cache is not None:
        cache.put(key, best, ms, trials)
    return best
