"""Tropical variable elimination with counting tuples (oracle; test only).

What it computes (Sec. II):
  * local tensors: on every edge the bond tensor holding the negative bond
    energy, [[J, -J], [-J, J]] for Ising (Sec. II), J * delta(a, b) for the
    Potts glass; on every spin the vertex ("dot") tensor holding h_i on state
    +1 and -h_i on state -1 (zero when h vanishes, where it reduces to the
    tropical copy tensor);
  * contraction under the tropical algebra of Eq. 2 gives
    V = max_sigma (-E(sigma)), so E_min = -V (Sec. II);
  * with (x, n) counting tuples (Sec. II) the same contraction gives the
    number of ground states;
  * the ground state itself comes from backtracking the cached argmax of every
    maximisation (Sec. III, "caching intermediate contraction results and
    backtracking"), taking the first index on ties (the footnote in Sec. III).

The contraction is organised as bucket (variable) elimination, the max-sum
algorithm that the tropical network reduces to (Sec. III): for each spin in
the elimination order, every factor that mentions it is multiplied (values
added, counts multiplied) into one table over the union of their scopes, and
the spin is maximised out (counts of all maximising states summed).

Values are float64 (the float32 couplings are exact in float64).  Counts are
exact integers: int64 while a bound computed with Python integers shows the
next table cannot overflow, Python integers (object arrays) beyond that.
"""
import numpy as np

_INT64_SAFE = 1 << 62


class Factor:
    __slots__ = ("scope", "val", "cnt", "cmax")

    def __init__(self, scope, val, cnt, cmax):
        self.scope = list(scope)
        self.val = val
        self.cnt = cnt
        self.cmax = cmax


def local_tensors(inst, count=True):
    """Bond and vertex tensors of Sec. II, values = negative energies."""
    q = inst["q"]
    fs = []
    J = inst["J"].astype(np.float64)
    if q == 2:
        s = np.array([1.0, -1.0])
    for (u, v), j in zip(inst["edges"].tolist(), J.tolist()):
        if q == 2:
            val = j * np.outer(s, s)              # [[J, -J], [-J, J]]
        else:
            val = j * np.eye(q)                   # J delta(a, b)
        fs.append(Factor([u, v], val, np.ones((q, q), np.int64) if count else None, 1))
    h = inst.get("h")
    for i in range(inst["n"]):
        if q == 2:
            hi = 0.0 if h is None else float(h[i])
            val = hi * s                          # diag(h, -h) on the spin's index
        else:
            val = np.zeros(q)
        fs.append(Factor([i], val, np.ones(q, np.int64) if count else None, 1))
    return fs


def min_fill_order(inst):
    """Greedy min-fill elimination order on the interaction graph (ties: degree, id)."""
    n = inst["n"]
    adj = [set() for _ in range(n)]
    for u, v in inst["edges"].tolist():
        adj[u].add(v)
        adj[v].add(u)
    alive = set(range(n))
    order = []
    while alive:
        best = None
        for v in alive:
            nb = list(adj[v])
            fill = 0
            for a in range(len(nb)):
                for b in range(a + 1, len(nb)):
                    if nb[b] not in adj[nb[a]]:
                        fill += 1
            key = (fill, len(nb), v)
            if best is None or key < best[0]:
                best = (key, v)
        v = best[1]
        nb = list(adj[v])
        for a in nb:
            adj[a].discard(v)
            adj[a].update(x for x in nb if x != a)
        alive.discard(v)
        order.append(v)
    return order


def _aligned(f, union, q, arr):
    """View a factor's table on the axes of ``union`` (size-1 axes where absent)."""
    pos = [union.index(x) for x in f.scope]
    perm = np.argsort(pos)
    t = np.transpose(arr, perm)
    shape = [q if x in f.scope else 1 for x in union]
    return t.reshape(shape)


def solve(inst, order=None, count=True, config=True, max_eliminations=None):
    """Contract the instance's tropical network by variable elimination.

    Returns dict(E=float E_min, count=int or None, state=int8 array of state
    indices or None, width=largest table scope).
    ``order`` is a spin sequence; spins it leaves out are eliminated afterwards
    in min-fill order.  ``max_eliminations`` stops after that many spins and
    returns only dict(eliminated=k, width=...) (used to time a bounded sample).
    """
    return solve_factors(inst, local_tensors(inst, count), order, count, config,
                         max_eliminations)


def solve_factors(inst, factors, order=None, count=True, config=True, max_eliminations=None):
    """Variable elimination over given factors (values = negative costs).

    ``inst`` supplies n, q and the interaction graph (edges) for the min-fill
    completion of ``order``; ``factors`` is a list of Factor whose counts are
    ones (or None without counting).  Same results as ``solve``.
    """
    n, q = inst["n"], inst["q"]
    if order is None:
        order = min_fill_order(inst)
    order = [int(v) for v in order]
    seen = set(order)
    if len(seen) != len(order):
        raise ValueError("elimination order repeats a spin")
    order += [v for v in min_fill_order(inst) if v not in seen]

    trace = []
    width = 0
    for step, v in enumerate(order):
        if max_eliminations is not None and step >= max_eliminations:
            return dict(eliminated=step, width=width)
        bucket = [f for f in factors if v in f.scope]
        rest = [f for f in factors if v not in f.scope]
        others = sorted(set(x for f in bucket for x in f.scope) - {v})
        union = [v] + others
        width = max(width, len(union))
        shape = (q,) * len(union)
        val = np.zeros(shape)
        for f in bucket:
            val = val + _aligned(f, union, q, f.val)          # (.) = +
        m = val.max(axis=0)                                    # (+) = max over v
        if config:
            trace.append((v, others, np.argmax(val, axis=0).astype(np.uint8)))
        if count:
            bound = q
            for f in bucket:
                bound *= f.cmax
            big = bound >= _INT64_SAFE
            cnt = np.ones(shape, dtype=object if big else np.int64)
            for f in bucket:
                c = f.cnt.astype(object) if big and f.cnt.dtype != object else f.cnt
                cnt = cnt * _aligned(f, union, q, c)           # counts multiply
            tie = val == m[None, ...]
            newc = np.where(tie, cnt, 0).sum(axis=0)           # ties add counts
            if not isinstance(newc, np.ndarray):
                newc = np.asarray(newc, dtype=object if big else np.int64)
            if newc.dtype != object:
                newc = newc.astype(np.int64)
            cmax = int(newc.max()) if newc.size else 0
        else:
            newc, cmax = None, 0
        rest.append(Factor(others, m, newc, cmax))
        factors = rest

    V = 0.0
    total = 1
    for f in factors:                 # only scalars are left
        assert not f.scope
        V += float(f.val)
        if count:
            total *= int(f.cnt)
    state = None
    if config:
        state = np.full(n, -1, dtype=np.int64)
        for v, others, arg in reversed(trace):
            idx = tuple(int(state[x]) for x in others)
            state[v] = int(arg[idx]) if others else int(arg)
        state = state.astype(np.int8)
    return dict(E=-V, count=total if count else None, state=state, width=width)
