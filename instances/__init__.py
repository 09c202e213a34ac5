"""Seeded synthetic spin-glass instances.

This module only draws random couplings and builds graphs; it holds none of the
contraction arithmetic, so both the CPU oracle and the CUDA path may use it.

An instance is a plain dict:

    n      number of spins
    q      states per spin (2 = Ising, 3 = Potts)
    edges  int32 array (n_edges, 2), 0-based spin ids, u != v, no duplicates
    J      float32 array (n_edges,)   coupling of each edge
    h      float32 array (n) or None  local field (Ising only)
    name   short description with the sizes
    seed   the seed the couplings were drawn with

Energy conventions (the arithmetic itself lives elsewhere):
  Ising (Eq. 1):  E(sigma) = -sum_e J_e sigma_u sigma_v - sum_i h_i sigma_i,
                  sigma in {+1, -1}; state index 0 <-> +1, index 1 <-> -1.
  Potts (App. C, with the sign convention of the 18x18 Potts-glass workload):
                  E(s) = -sum_e J_e delta(s_u, s_v), s in {0, 1, 2}.

Gaussian couplings are drawn in float64 and rounded to float32: the float32
values are the instance.  +-J couplings are +1/-1 with probability 1/2 each.
"""
from __future__ import annotations

import hashlib

import numpy as np

__all__ = [
    "square_lattice", "chimera", "random_regular3", "potts_square",
    "mixed_square_batch", "planted", "ferromagnet", "instance_digest",
    "square_sweep_order", "chimera_sweep_order", "potts_planted",
    "cubic_lattice", "cubic_edges", "max2sat_regular3", "max2sat_planted",
]


def _couplings(rng, m, kind):
    if kind == "pm1":
        return np.where(rng.integers(0, 2, size=m) == 0, 1.0, -1.0).astype(np.float32)
    if kind == "gauss":
        return rng.standard_normal(m).astype(np.float32)
    if kind == "zero":
        return np.zeros(m, np.float32)
    raise ValueError(f"unknown coupling kind {kind!r}")


def _fields(rng, n, sigma):
    if sigma is None or sigma == 0:
        return None
    return (sigma * rng.standard_normal(n)).astype(np.float32)


def square_edges(L, W=None):
    """Open-boundary L x W square lattice; spin (r, c) has id r*W + c.

    Edges are listed spin by spin in id order: first the bond to the right
    neighbour, then the bond to the one below.
    """
    W = L if W is None else W
    e = []
    for r in range(L):
        for c in range(W):
            i = r * W + c
            if c + 1 < W:
                e.append((i, i + 1))
            if r + 1 < L:
                e.append((i, i + W))
    return np.asarray(e, dtype=np.int32).reshape(-1, 2)


def square_lattice(L, W=None, coupling="pm1", field_sigma=None, seed=0):
    """L x W open square-lattice Ising spin glass (Sec. IV, Fig. 1)."""
    W = L if W is None else W
    rng = np.random.default_rng(seed)
    edges = square_edges(L, W)
    J = _couplings(rng, len(edges), coupling)
    h = _fields(rng, L * W, field_sigma)
    return dict(n=L * W, q=2, edges=edges, J=J, h=h, seed=seed,
                name=f"square{L}x{W}-{coupling}" + (f"-h{field_sigma}" if h is not None else ""))


def square_sweep_order(L, W=None):
    """Row-by-row spin sequence of an L x W lattice (the circuit sweep of Fig. 1b)."""
    W = L if W is None else W
    return np.arange(L * W, dtype=np.int32)


def cubic_edges(L, W=None, H=None):
    """Open-boundary L x W x H cubic lattice; spin (x, y, z) has id (x*W + y)*H + z.

    Edges are listed spin by spin in id order: the bond along z, then along y,
    then along x (each only where the neighbour exists).
    """
    W = L if W is None else W
    H = L if H is None else H
    e = []
    for x in range(L):
        for y in range(W):
            for z in range(H):
                i = (x * W + y) * H + z
                if z + 1 < H:
                    e.append((i, i + 1))
                if y + 1 < W:
                    e.append((i, i + H))
                if x + 1 < L:
                    e.append((i, i + W * H))
    return np.asarray(e, dtype=np.int32).reshape(-1, 2)


def cubic_lattice(L, W=None, H=None, coupling="pm1", field_sigma=None, seed=0):
    """L x W x H open cubic-lattice Ising spin glass (the 3D workload of Sec. IV)."""
    W = L if W is None else W
    H = L if H is None else H
    rng = np.random.default_rng(seed)
    edges = cubic_edges(L, W, H)
    J = _couplings(rng, len(edges), coupling)
    h = _fields(rng, L * W * H, field_sigma)
    return dict(n=L * W * H, q=2, edges=edges, J=J, h=h, seed=seed,
                name=f"cubic{L}x{W}x{H}-{coupling}" + (f"-h{field_sigma}" if h is not None else ""))


def chimera_edges(L):
    """Chimera graph of L x L K_{4,4} unit cells (Sec. IV, Fig. 2a).

    Cell (i, j) holds spins 8*(i*L+j) + k, k = 0..7.  Spins k = 0..3 form the
    half coupled vertically (spin k of cell (i, j) to spin k of cell (i+1, j)),
    spins k = 4..7 the half coupled horizontally (to cell (i, j+1)).  Inside a
    cell every spin of one half couples to every spin of the other (16 edges).
    L = 8 gives 512 spins and 1024 + 224 + 224 = 1472 couplers.
    """
    e = []
    for i in range(L):
        for j in range(L):
            b = 8 * (i * L + j)
            for a in range(4):
                for c in range(4):
                    e.append((b + a, b + 4 + c))
            if i + 1 < L:
                bn = 8 * ((i + 1) * L + j)
                for a in range(4):
                    e.append((b + a, bn + a))
            if j + 1 < L:
                bn = 8 * (i * L + j + 1)
                for a in range(4):
                    e.append((b + 4 + a, bn + 4 + a))
    return np.asarray(e, dtype=np.int32).reshape(-1, 2)


def chimera_sweep_order(L):
    """Spin sequence sweeping the chimera by cell rows: for each row of cells,
    first every spin of the horizontally coupled halves, then every spin of
    the vertically coupled halves (keeps about 4L + 1 spins live)."""
    seq = []
    for i in range(L):
        for j in range(L):
            seq += [8 * (i * L + j) + k for k in range(4, 8)]
        for j in range(L):
            seq += [8 * (i * L + j) + k for k in range(4)]
    return np.asarray(seq, dtype=np.int32)


def chimera(L, coupling="pm1", seed=0):
    rng = np.random.default_rng(seed)
    edges = chimera_edges(L)
    J = _couplings(rng, len(edges), coupling)
    return dict(n=8 * L * L, q=2, edges=edges, J=J, h=None, seed=seed,
                name=f"chimera{L}x{L}-{coupling}")


def random_regular3_edges(N, rng, max_tries=100000):
    """Random 3-regular graph by the pairing (configuration) model.

    3N stubs are matched by a uniformly random perfect matching; a matching
    with a self-loop or a repeated edge is thrown away and redrawn whole.
    """
    if (3 * N) % 2:
        raise ValueError("3N must be even")
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(N), 3)
        perm = rng.permutation(3 * N)
        pairs = stubs[perm].reshape(-1, 2)
        u = np.minimum(pairs[:, 0], pairs[:, 1])
        v = np.maximum(pairs[:, 0], pairs[:, 1])
        if np.any(u == v):
            continue
        key = u.astype(np.int64) * N + v
        if len(np.unique(key)) != len(key):
            continue
        order = np.argsort(key)
        return np.stack([u[order], v[order]], axis=1).astype(np.int32)
    raise RuntimeError("pairing model did not produce a simple graph")


def random_regular3(N, coupling="gauss", seed=0):
    rng = np.random.default_rng(seed)
    edges = random_regular3_edges(N, rng)
    J = _couplings(rng, len(edges), coupling)
    return dict(n=N, q=2, edges=edges, J=J, h=None, seed=seed,
                name=f"rrg3-N{N}-{coupling}")


def max2sat_regular3(N, seed=0):
    """Random Max-2-SAT instance on a random 3-regular graph (App. D).

    Every edge (u, v) of a pairing-model 3-regular graph on N variables is one
    clause l_u OR l_v; each literal is negated independently with
    probability 1/2.  Returned as a dict:

        n        number of variables
        clauses  int32 array (m, 2) of literals: +(i+1) for x_i, -(i+1) for NOT x_i
        name, seed
    """
    rng = np.random.default_rng(seed)
    edges = random_regular3_edges(N, rng)
    neg = rng.integers(0, 2, size=edges.shape) == 1
    lits = np.where(neg, -(edges + 1), edges + 1).astype(np.int32)
    return dict(n=N, clauses=lits, seed=seed, name=f"max2sat-rrg3-N{N}")


def max2sat_planted(sat, seed=0):
    """A satisfiable variant of a Max-2-SAT instance: for a random assignment
    tau, every clause that tau violates gets its first literal negated, so tau
    satisfies all clauses.  Returns (instance, tau as int8 array of 0/1 with
    1 = true)."""
    rng = np.random.default_rng(seed)
    tau = rng.integers(0, 2, size=sat["n"]).astype(np.int8)
    lits = sat["clauses"].copy()
    var = np.abs(lits) - 1
    true_lit = np.where(lits > 0, tau[var] == 1, tau[var] == 0)
    violated = ~true_lit[:, 0] & ~true_lit[:, 1]
    lits[violated, 0] = -lits[violated, 0]
    return dict(sat, clauses=lits, name=sat["name"] + "-planted"), tau


def potts_square(L, W=None, coupling="gauss", seed=0):
    """q = 3 Potts glass on an open L x W square lattice (App. C)."""
    W = L if W is None else W
    rng = np.random.default_rng(seed)
    edges = square_edges(L, W)
    J = _couplings(rng, len(edges), coupling)
    return dict(n=L * W, q=3, edges=edges, J=J, h=None, seed=seed,
                name=f"potts3-square{L}x{W}-{coupling}")


def mixed_square_batch(B, Lmin=8, Lmax=20, coupling="pm1", seed=0):
    """B square +-J lattices with L uniform in [Lmin, Lmax], instance k seeded seed+1+k."""
    rng = np.random.default_rng(seed)
    Ls = rng.integers(Lmin, Lmax + 1, size=B)
    return [square_lattice(int(L), coupling=coupling, seed=seed + 1 + k) for k, L in enumerate(Ls)]


def planted(inst, seed=0):
    """Mattis (gauge-transformed ferromagnet) version of an instance.

    J_uv -> |J_uv| tau_u tau_v for a random tau in {+1,-1}^n, fields dropped.
    Its ground states are exactly tau and -tau on a connected graph.
    Returns (instance, tau as int8 array of +-1).
    """
    rng = np.random.default_rng(seed)
    tau = np.where(rng.integers(0, 2, size=inst["n"]) == 0, 1, -1).astype(np.int8)
    e = inst["edges"]
    J = (np.abs(inst["J"]) * tau[e[:, 0]] * tau[e[:, 1]]).astype(np.float32)
    out = dict(inst, J=J, h=None, name=inst["name"] + "-planted")
    return out, tau


def potts_planted(inst, seed=0):
    """Potts glass whose couplings are satisfied by a random colouring tau:
    J_uv -> |J_uv| if tau_u == tau_v else -|J_uv|.  tau is a ground state and
    E_min = -sum of the positive couplings.  Returns (instance, tau)."""
    rng = np.random.default_rng(seed)
    tau = rng.integers(0, inst["q"], size=inst["n"]).astype(np.int8)
    e = inst["edges"]
    same = tau[e[:, 0]] == tau[e[:, 1]]
    J = np.where(same, np.abs(inst["J"]), -np.abs(inst["J"])).astype(np.float32)
    return dict(inst, J=J, name=inst["name"] + "-planted"), tau


def ferromagnet(inst):
    """Same graph with every coupling replaced by its absolute value, no fields."""
    return dict(inst, J=np.abs(inst["J"]).astype(np.float32), h=None,
                name=inst["name"] + "-ferro")


def instance_digest(inst):
    """sha256 over the instance's arrays; pins a stored expected value to its input."""
    m = hashlib.sha256()
    if "clauses" in inst:
        m.update(np.int64(inst["n"]).tobytes())
        m.update(np.ascontiguousarray(inst["clauses"], dtype=np.int32).tobytes())
        return m.hexdigest()
    m.update(np.int64(inst["n"]).tobytes())
    m.update(np.int64(inst["q"]).tobytes())
    m.update(np.ascontiguousarray(inst["edges"], dtype=np.int32).tobytes())
    m.update(np.ascontiguousarray(inst["J"], dtype=np.float32).tobytes())
    if inst.get("h") is not None:
        m.update(np.ascontiguousarray(inst["h"], dtype=np.float32).tobytes())
    return m.hexdigest()
