"""The batch autotuner's search (host logic, CPU): coordinate descent over
the CTAs per SM of each stage and the schedule knobs (blocks per integration
CTA, scattered walks) keeps a candidate only when it gains at least
min_gain, ends on the best setting it timed and leaves the batch set to it.
The timing and the batch are replaced by a fake with a known cost."""

import paper_1708_00783_gb300.autotune as at

N = at.ITM_BATCH_STAGES
K = at.ITM_BATCH_KNOBS
DEFAULT = [0] * N + [1, 0, 0]


class FakeBatch:
    def __init__(self, cost):
        self.setting = list(DEFAULT)
        self.cost = cost
        self.timed = []


def install(monkeypatch, fb):
    monkeypatch.setattr(at, "itm_batch_set_tuning", lambda b, v: fb.setting.__setitem__(slice(0, N), list(v)))
    monkeypatch.setattr(at, "itm_batch_set_schedule", lambda b, v: fb.setting.__setitem__(slice(N, N + K), list(v)))
    monkeypatch.setattr(at, "itm_batch_get_tuning", lambda b: list(fb.setting[:N]))

    def time_steps(step, reps, stream):
        t = fb.cost(fb.setting)
        fb.timed.append((list(fb.setting), t))
        return t

    monkeypatch.setattr(at, "time_steps", time_steps)


def test_descent_finds_a_separable_optimum(monkeypatch):
    target = [2, 1, 4, 8, 1, 4][:N] + [0] * max(0, N - 6) + [4, 1, 0]
    fb = FakeBatch(lambda v: 1.0 + sum((1.0 if c != t else 0.0) * (0.1 * (s + 1)) for s, (c, t) in
                                       enumerate(zip(v, target))))
    install(monkeypatch, fb)
    cur, best, log, final = at.tune_batch(object(), lambda: None, None)
    assert cur == target and final == target[:N] and fb.setting == target
    assert best == 1.0
    assert min(t for _, t in fb.timed) == best


def test_gains_below_min_gain_are_not_taken(monkeypatch):
    # every non-default setting is 0.5% faster: below the 1% threshold
    fb = FakeBatch(lambda v: 1.0 - (0.005 if v != DEFAULT else 0.0))
    install(monkeypatch, fb)
    cur, best, log, final = at.tune_batch(object(), lambda: None, None, min_gain=0.01)
    assert cur == DEFAULT and best == 1.0 and fb.setting == DEFAULT
    # the default, then each stage's four other CTA counts and each knob's other values
    assert len(log) == 1 + N * 4 + (2 + 1 + 1)


def test_each_stage_is_tuned_with_the_others_at_their_best_so_far(monkeypatch):
    # stage 1's best value depends on stage 0's: coordinate descent sees
    # stage 0 already moved when it tries stage 1
    def cost(v):
        return 10.0 - (3.0 if v[0] == 4 else 0.0) - (2.0 if (v[0] == 4 and v[1] == 8) else 0.0)

    fb = FakeBatch(cost)
    install(monkeypatch, fb)
    cur, best, _, _ = at.tune_batch(object(), lambda: None, None)
    assert cur[:2] == [4, 8] and best == 5.0
