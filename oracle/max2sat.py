"""Max-2-SAT as a tropical network (oracle; test only).

App. D counts the optimal assignments of Max-2-SAT instances on random
3-regular graphs with the same machinery as the spin glasses: the cost of an
assignment x in {0, 1}^n (1 = true) is the number of violated clauses, each
clause l_u OR l_v contributes one local tensor over its two variables, and the
network holds negative costs, so its tropical contraction gives
-min_x cost(x) and the counting tuples of Sec. II the number of minimisers.

Literals are signed 1-based variable ids: +(i+1) is x_i, -(i+1) is NOT x_i.
Here the tensors are built straight from the clauses (a 2 x 2 table that is
-1 at the one violating pair of values and 0 elsewhere); nothing passes
through Ising couplings.
"""
import numpy as np

from .elimination import Factor, solve_factors


def _lit(l):
    """(variable, value of x that makes the literal true)."""
    return abs(int(l)) - 1, (1 if l > 0 else 0)


def cost(sat, states):
    """Violated clauses of each assignment; states is (k, n) of 0/1 (1 = true)."""
    states = np.atleast_2d(np.asarray(states, dtype=np.int64))
    lits = np.asarray(sat["clauses"], dtype=np.int64)
    var = np.abs(lits) - 1
    want = (lits > 0).astype(np.int64)
    ok = states[:, var] == want[None, :, :]               # (k, m, 2): literal true
    return np.sum(~(ok[:, :, 0] | ok[:, :, 1]), axis=1)


def brute_force(sat):
    """The plain definition: every assignment, min cost and its multiplicity."""
    n = sat["n"]
    if n > 22:
        raise ValueError("brute force is for n <= 22")
    best, cnt, first = None, 0, None
    chunk = 1 << 16
    for start in range(0, 1 << n, chunk):
        idx = np.arange(start, min(start + chunk, 1 << n), dtype=np.int64)
        states = (idx[:, None] >> np.arange(n)[None, :]) & 1
        c = cost(sat, states)
        m = int(c.min())
        if best is None or m < best:
            best, cnt, first = m, int(np.sum(c == m)), states[int(np.argmax(c == m))]
        elif m == best:
            cnt += int(np.sum(c == m))
    return dict(E=best, count=cnt, state=first.astype(np.int8))


def clause_tensors(sat, count=True):
    """One factor per clause (-1 at the violating values) plus a zero factor
    per variable, so that variables in no clause still count twice."""
    n = sat["n"]
    fs = []
    for l1, l2 in np.asarray(sat["clauses"]).tolist():
        (u, tu), (v, tv) = _lit(l1), _lit(l2)
        if u == v:
            val = np.zeros(2)
            for a in range(2):
                if a != tu and a != tv:
                    val[a] = -1.0
            fs.append(Factor([u], val, np.ones(2, np.int64) if count else None, 1))
            continue
        val = np.zeros((2, 2))
        val[1 - tu, 1 - tv] = -1.0
        fs.append(Factor([u, v], val, np.ones((2, 2), np.int64) if count else None, 1))
    for i in range(n):
        fs.append(Factor([i], np.zeros(2), np.ones(2, np.int64) if count else None, 1))
    return fs


def interaction_graph(sat):
    lits = np.asarray(sat["clauses"], dtype=np.int64)
    var = np.abs(lits) - 1
    pairs = {(min(a, b), max(a, b)) for a, b in var.tolist() if a != b}
    e = np.asarray(sorted(pairs), dtype=np.int32).reshape(-1, 2)
    return dict(n=sat["n"], q=2, edges=e)


def solve(sat, order=None, count=True, config=True):
    """Min cost, number of optimal assignments and one of them (0/1, 1 = true)."""
    g = interaction_graph(sat)
    r = solve_factors(g, clause_tensors(sat, count), order, count, config)
    return dict(E=int(round(r["E"])), count=r["count"], state=r["state"], width=r["width"])
