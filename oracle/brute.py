"""Exhaustive enumeration (oracle; test infrastructure only).

The plain definition of what the contraction computes (Sec. II):
E_min = min over all q^N states of E, the degeneracy is the number of states
that reach it, and a ground state is any one of them.
"""
import numpy as np

from .energy import energies_of


def all_states(n, q, start, stop):
    """States with mixed-radix rank start..stop-1; spin 0 is the slowest digit."""
    r = np.arange(start, stop, dtype=np.int64)
    out = np.empty((len(r), n), dtype=np.int8)
    for i in range(n - 1, -1, -1):
        out[:, i] = r % q
        r //= q
    return out


def brute_force(inst, chunk=1 << 16, keep_states=True):
    """Return dict(E=E_min, count=int, states=array of all ground states).

    Energies are compared with exact float64 equality; use integral couplings
    (or symmetric partners, which give bit-identical sums) when counts matter.
    """
    n, q = inst["n"], inst["q"]
    total = q ** n
    if total > (1 << 24):
        raise ValueError(f"{total} states is too many for brute force")
    best, count, states = np.inf, 0, []
    for s in range(0, total, chunk):
        st = all_states(n, q, s, min(total, s + chunk))
        E = energies_of(inst, st)
        m = E.min()
        if m < best:
            best, count, states = m, 0, []
        if m == best:
            sel = E == best
            count += int(sel.sum())
            if keep_states:
                states.append(st[sel])
    gs = np.concatenate(states) if keep_states and states else None
    return dict(E=float(best), count=count, states=gs)
