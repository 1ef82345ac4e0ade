"""Host logic of the attempts loop (api.plan_attempts, Sec. 5.2): each attempt
plans only the problems no earlier attempt solved, with that attempt's seeds;
a problem keeps the best trajectory of the attempt that solved it."""
import numpy as np
import pytest
import torch

from paper_2410_16727_gb300 import api

P, S, T = 6, 3, 4
# attempt (1-based) whose plan solves each problem, 0: never; and the best seed then
SOLVES_AT = np.array([1, 2, 0, 3, 1, 2])
BEST_SEED = np.array([2, 0, 0, 1, 1, 2])


def _fake():
    calls = []

    def seed_fn(attempt, problems):
        # seed value encodes (attempt, problem, seed index) so the result can be traced
        x = np.zeros((len(problems), S, T, 7), np.float32)
        for i, p in enumerate(problems):
            for s in range(S):
                x[i, s] = 100 * attempt + 10 * p + s
        return x

    def plan_fn(problems, seeds):
        calls.append((len(calls) + 1, problems.copy()))
        a = len(calls)
        best = np.where(SOLVES_AT[problems] == a, BEST_SEED[problems], -1)
        cost = seeds[:, :, 0, 0] * 0.5
        return {"traj": torch.as_tensor(seeds), "cost": torch.as_tensor(cost),
                "success": torch.as_tensor((best >= 0)[:, None] & (np.arange(S)[None] == best[:, None])),
                "best": torch.as_tensor(best.astype(np.int32))}

    return plan_fn, seed_fn, calls


@pytest.mark.parametrize("n_attempts", [1, 2, 3, 5])
def test_attempts_plan_only_unsolved_problems(n_attempts):
    plan_fn, seed_fn, calls = _fake()
    r = api.plan_attempts(plan_fn, seed_fn, P, n_attempts)
    want_att = np.where((SOLVES_AT > 0) & (SOLVES_AT <= n_attempts), SOLVES_AT, 0)
    np.testing.assert_array_equal(r["attempts"], want_att)
    np.testing.assert_array_equal(r["solved"], want_att > 0)
    # attempt a sees exactly the problems unsolved after a - 1 attempts; the loop stops early when none is left
    for a, probs in calls:
        np.testing.assert_array_equal(probs, np.nonzero((SOLVES_AT == 0) | (SOLVES_AT >= a))[0])
    assert len(calls) == n_attempts              # problem 2 is never solved, so every attempt runs
    for p in range(P):
        if want_att[p]:
            v = 100 * want_att[p] + 10 * p + BEST_SEED[p]
            assert np.all(r["traj"][p] == v) and r["cost"][p] == pytest.approx(0.5 * v)
        else:
            assert np.isnan(r["traj"][p]).all() and np.isnan(r["cost"][p])


def test_loop_ends_when_everything_is_solved():
    calls = []

    def plan_fn(problems, seeds):
        calls.append(problems)
        n = len(problems)
        return {"traj": torch.zeros(n, 1, T, 7), "cost": torch.zeros(n, 1),
                "success": torch.ones(n, 1, dtype=torch.bool), "best": torch.zeros(n, dtype=torch.int32)}

    r = api.plan_attempts(plan_fn, lambda a, p: np.zeros((len(p), 1, T, 7), np.float32), 4, 10)
    assert len(calls) == 1 and r["solved"].all() and (r["attempts"] == 1).all()


def test_bad_arguments():
    with pytest.raises(ValueError):
        api.plan_attempts(None, None, 3, 0)
