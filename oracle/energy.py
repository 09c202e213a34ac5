"""Direct energy evaluation (oracle; test infrastructure only).

Ising, Eq. 1:  E(sigma) = -sum_{i<j} J_ij sigma_i sigma_j - sum_i h_i sigma_i.
State index a in {0, 1} maps to sigma = +1, -1, following the layout of the
bond matrix [[J, -J], [-J, J]] of Sec. II.

Potts (q = 3): E(s) = -sum_e J_e delta(s_u, s_v).  This is the sign
convention of the 18x18 Potts-glass workload; App. C writes the same model as
H = sum J M_{s_u s_v} with M = 3/2 delta - 1/2, which has the same ground
states under J -> -J.
"""
import numpy as np


def spin_value(a):
    """State index 0 -> +1, 1 -> -1 (Sec. II bond-matrix layout)."""
    return 1 - 2 * np.asarray(a, dtype=np.int64)


def energies_of(inst, states):
    """Energies in float64 of a batch of states, shape (B, n) of state indices."""
    states = np.asarray(states)
    e = inst["edges"]
    J = inst["J"].astype(np.float64)
    u = states[:, e[:, 0]]
    v = states[:, e[:, 1]]
    if inst["q"] == 2:
        s = spin_value(states).astype(np.float64)
        E = -(s[:, e[:, 0]] * s[:, e[:, 1]]) @ J
        if inst.get("h") is not None:
            E = E - s @ inst["h"].astype(np.float64)
        return E
    return -((u == v).astype(np.float64) @ J)


def energy(inst, state):
    """Energy of one state (array of n state indices)."""
    return float(energies_of(inst, np.asarray(state)[None, :])[0])
