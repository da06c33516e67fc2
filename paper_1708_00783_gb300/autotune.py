"""Autotuner for the batched per-frame path.

Searches, by coordinate descent, the launch shape of each persistent batch
stage (CTAs per SM, itm_batch_set_tuning) together with the batch's
schedule (itm_batch_set_schedule: blocks per integration CTA, scattered or
in-order tile walks of the enumeration and the raycast), timing whole batch
steps with CUDA events on the stream they run on.  Every candidate is timed
on the work the caller supplies (one batch step per call of `step`), after
one untimed step that captures the CUDA graph for the candidate.  The
caller decides what the steps are: the bench tunes on frames and scenes of
their own and then times the chosen setting and the default on other
frames.
"""

from __future__ import annotations

from . import (ITM_BATCH_KNOBS, ITM_BATCH_STAGES, itm_batch_get_tuning, itm_batch_set_schedule,
               itm_batch_set_tuning)

STAGE_NAMES = ["enumerate", "commit", "visible", "integrate", "range", "raycast"]
KNOB_NAMES = ["integrate_blocks_per_cta", "enumerate_scatter", "raycast_scatter"]
CTA_CANDIDATES = (0, 1, 2, 4, 8)
KNOB_CANDIDATES = ((1, 2, 4), (0, 1), (0, 1))
DEFAULT_SCHEDULE = [1, 0, 0]


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


def apply(batch, setting):
    """setting: CTAs per SM of each stage, then the schedule knobs."""
    itm_batch_set_tuning(batch, setting[:ITM_BATCH_STAGES])
    itm_batch_set_schedule(batch, setting[ITM_BATCH_STAGES:])


def tune_batch(batch, step, stream, candidates=CTA_CANDIDATES, passes=1, reps=3, min_gain=0.01):
    """Returns (setting, best ms per step, log of trials, grid sizes); the
    setting is the CTAs per SM of each stage followed by the schedule knobs,
    and the batch is left set to it."""
    cur = [0] * ITM_BATCH_STAGES + list(DEFAULT_SCHEDULE)
    apply(batch, cur)
    best = time_steps(step, reps, stream)
    log = [("default", list(cur), best)]
    coords = [(st, STAGE_NAMES[st], candidates) for st in range(ITM_BATCH_STAGES)]
    coords += [(ITM_BATCH_STAGES + k, KNOB_NAMES[k], KNOB_CANDIDATES[k]) for k in range(ITM_BATCH_KNOBS)]
    for _ in range(passes):
        for idx, name, cands in coords:
            for c in cands:
                if c == cur[idx]:
                    continue
                trial = list(cur)
                trial[idx] = c
                apply(batch, trial)
                t = time_steps(step, reps, stream)
                log.append((name, list(trial), t))
                if t < best * (1.0 - min_gain):
                    best, cur = t, trial
    apply(batch, cur)
    return cur, best, log, itm_batch_get_tuning(batch)
