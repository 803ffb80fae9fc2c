"""Autotuner: pick the gate-kernel configuration for a workload by timing.

Candidates vary how a gate's work is split (one warp per gate with windows
of 128 or 352 transitions per pin of 3-input cells, longer for fewer
inputs, i.e. the event chunk size; or one lane per time segment with a
given segment size) and the CTA shape.  Each candidate builds
the caller's run, runs it once to warm up, then times `reruns` evaluations
with the library's own device timer and scores the candidate by the median
(an odd count, so the median is one measured run); the fastest configuration
is left applied to the context and returned.  Results are identical for every
candidate (all variants are parity-tested), so tuning only affects speed.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import gls as _g

DEFAULT_CANDIDATES = [
    {"kernel": "wide", "warps_per_cta": 4},
    {"kernel": "wide", "warps_per_cta": 2},
    {"kernel": "windowed", "warps_per_cta": 4},
    {"kernel": "windowed", "warps_per_cta": 2},
    {"kernel": "segmented", "warps_per_cta": 4, "segment": 32},
    {"kernel": "segmented", "warps_per_cta": 4, "segment": 128},
]


@dataclass
class TuneResult:
    best: dict
    timings_ms: list          # (candidate, median ms) in trial order


def apply(ctx, cand: dict):
    ctx.set_kernel(cand["kernel"])
    ctx.set_option(_g.GLS_OPT_WARPS_PER_CTA, cand.get("warps_per_cta", 4))
    if "segment" in cand:
        ctx.set_option(_g.GLS_OPT_SEGMENT, cand["segment"])


def autotune(ctx, build_run, candidates=None, reruns: int = 3) -> TuneResult:
    """build_run() -> run id of a freshly created run of the workload (it is
    released here).  Returns the fastest candidate, applied to ctx."""
    if reruns < 1 or reruns % 2 == 0:
        raise ValueError("reruns must be a positive odd count (the score is their median)")
    cands = candidates or DEFAULT_CANDIDATES
    times = []
    for cand in cands:
        apply(ctx, cand)
        rid = build_run()
        ctx.run_stats(rid)
        ms = []
        for _ in range(reruns):
            ctx.rerun(rid)
            ms.append(ctx.run_stats(rid).kernel_ms)
        ctx.release(rid)
        ms.sort()
        times.append((cand, ms[len(ms) // 2]))
    best = min(times, key=lambda x: x[1])[0]
    apply(ctx, best)
    return TuneResult(best, times)
