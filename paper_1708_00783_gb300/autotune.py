"""Autotuner for the batched per-frame path.

Searches the CTAs per SM of each persistent batch stage (itm_batch_set_tuning)
by coordinate descent, timing whole batch steps with CUDA events on the
stream they run on.  Every candidate is timed on the work the caller supplies
(one batch step per call of `step`), after one untimed step that captures the
CUDA graph for the candidate's launch shapes.
"""

from __future__ import annotations

from . import ITM_BATCH_STAGES, itm_batch_get_tuning, itm_batch_set_tuning

STAGE_NAMES = ["enumerate", "commit", "visible", "integrate", "range", "raycast"]


def time_steps(step, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step()
    a.record(stream)
    for _ in range(reps):
        step()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune_batch(batch, step, stream, candidates=(0, 1, 2, 4, 8), passes=1, reps=3, min_gain=0.01):
    """Returns (ctas_per_sm per stage, best ms per step, log of trials)."""
    cur = [0] * ITM_BATCH_STAGES
    itm_batch_set_tuning(batch, cur)
    best = time_steps(step, reps, stream)
    log = [("default", list(cur), best)]
    for _ in range(passes):
        for st in range(ITM_BATCH_STAGES):
            for c in candidates:
                if c == cur[st]:
                    continue
                trial = list(cur)
                trial[st] = c
                itm_batch_set_tuning(batch, trial)
                t = time_steps(step, reps, stream)
                log.append((STAGE_NAMES[st], list(trial), t))
                if t < best * (1.0 - min_gain):
                    best, cur = t, trial
    itm_batch_set_tuning(batch, cur)
    return cur, best, log, itm_batch_get_tuning(batch)
