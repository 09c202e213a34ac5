"""Pins of the Max-2-SAT oracle (App. D): the cost of an assignment is the
number of violated clauses; contracting the clause network gives the minimum
cost and the number of optimal assignments.  CPU only."""
import numpy as np
import pytest

import instances as I
from oracle import max2sat as M


def _sat(n, clauses):
    return dict(n=n, clauses=np.asarray(clauses, np.int32).reshape(-1, 2), name="hand", seed=0)


def test_cost_by_hand():
    sat = _sat(3, [(1, 2), (-1, 3)])
    # x = (F, F, F): clause 1 has both literals false, clause 2 has NOT x1 true
    assert M.cost(sat, [0, 0, 0])[0] == 1
    # x = (T, F, F): clause 1 satisfied by x1, clause 2 has NOT x1 and x3 false
    assert M.cost(sat, [1, 0, 0])[0] == 1
    assert M.cost(sat, [1, 0, 1])[0] == 0
    assert M.cost(sat, [0, 1, 0])[0] == 0


def test_all_four_sign_patterns_on_one_pair():
    # every assignment of (x1, x2) violates exactly one of the four clauses
    sat = _sat(2, [(1, 2), (1, -2), (-1, 2), (-1, -2)])
    for r in (M.brute_force(sat), M.solve(sat)):
        assert (r["E"], r["count"]) == (1, 4)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_disjoint_clauses(k):
    # k clauses on disjoint pairs: each has 3 satisfying assignments of its pair
    sat = _sat(2 * k, [(2 * i + 1, -(2 * i + 2)) for i in range(k)])
    r = M.solve(sat)
    assert (r["E"], r["count"]) == (0, 3 ** k)


def test_free_variables_double_the_count():
    sat = _sat(5, [(1, 2)])
    r = M.solve(sat)
    assert (r["E"], r["count"]) == (0, 3 * 2 ** 3)


def test_implication_chain():
    # (NOT x_i OR x_{i+1}) for i < n: x is a monotone 0...01...1 string, n + 1 of them
    n = 9
    sat = _sat(n, [(-(i + 1), i + 2) for i in range(n - 1)])
    r = M.solve(sat)
    assert (r["E"], r["count"]) == (0, n + 1)


@pytest.mark.parametrize("N,seed", [(12, 0), (12, 1), (16, 2), (16, 3), (20, 5), (20, 7)])
def test_elimination_matches_brute_force(N, seed):
    sat = I.max2sat_regular3(N, seed=seed)
    b = M.brute_force(sat)
    rng = np.random.default_rng(seed)
    for order in (None, list(range(N)), rng.permutation(N).tolist()):
        r = M.solve(sat, order=order)
        assert (r["E"], r["count"]) == (b["E"], b["count"])
        assert M.cost(sat, r["state"])[0] == b["E"]


def test_some_small_instance_is_unsatisfiable():
    # the brute-force comparison above must include optimum > 0
    assert M.brute_force(I.max2sat_regular3(20, seed=5))["E"] >= 1


@pytest.mark.parametrize("N", [20, 60])
def test_planted_is_satisfiable(N):
    sat, tau = I.max2sat_planted(I.max2sat_regular3(N, seed=9), seed=4)
    assert M.cost(sat, tau)[0] == 0
    r = M.solve(sat)
    assert r["E"] == 0 and r["count"] >= 1
    assert M.cost(sat, r["state"])[0] == 0


def test_planted_clause_mistake_is_caught(monkeypatch):
    """A clause tensor that marks the wrong pair of values must break a pin."""
    orig = M.clause_tensors

    def wrong(sat, count=True):
        fs = orig(sat, count)
        for f in fs:
            if len(f.scope) == 2:
                f.val = f.val[::-1, :].copy()
        return fs

    monkeypatch.setattr(M, "clause_tensors", wrong)
    sat = I.max2sat_regular3(16, seed=2)
    r, b = M.solve(sat), M.brute_force(sat)
    assert (r["E"], r["count"]) != (b["E"], b["count"])
