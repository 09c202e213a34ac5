"""Pins for the CPU oracle: values fixed by the paper's definitions and by
mathematics, never by the oracle itself or by the CUDA path.

  * hand-derived golden examples (tests/golden/hand_examples.json, Eq. 1 / App. C)
  * brute force over all states against the elimination (Sec. II definition)
  * closed forms: ferromagnet, Mattis-planted glass, J = 0, frustrated rings,
    proper 3-colourings of paths and cycles (chromatic polynomials)
  * tree graphs against an independent leaf-to-root max-sum DP (Sec. III)
  * invariants: energy parity and even degeneracy of +-J glasses, Potts
    degeneracy divisible by 3, order independence, finite differences in h
  * the semiring products against path enumeration in a layered graph
  * a planted mistake in the oracle must be caught
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import instances as I
import oracle as O
from oracle import semiring as S

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _inst_from_case(c):
    return dict(n=c["n"], q=c["q"], edges=np.asarray(c["edges"], np.int32).reshape(-1, 2),
                J=np.asarray(c["J"], np.float32),
                h=None if c["h"] is None else np.asarray(c["h"], np.float32),
                name=c["name"], seed=0)


def _cases():
    with open(GOLD) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_golden_brute_force(case):
    inst = _inst_from_case(case)
    b = O.brute_force(inst)
    assert b["E"] == case["E"]
    assert b["count"] == case["count"]
    if case["ground_states"] is not None:
        got = sorted(map(tuple, b["states"].tolist()))
        assert got == sorted(map(tuple, case["ground_states"]))


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_golden_elimination(case):
    inst = _inst_from_case(case)
    s = O.solve(inst)
    assert s["E"] == case["E"]
    assert s["count"] == case["count"]
    assert O.energy(inst, s["state"]) == case["E"]
    if case["ground_states"] is not None:
        assert tuple(s["state"].tolist()) in set(map(tuple, case["ground_states"]))


def _random_small(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "square_pm":
        return I.square_lattice(3, 4, coupling="pm1", seed=seed)
    if kind == "square_gauss_h":
        return I.square_lattice(3, 3, coupling="gauss", field_sigma=0.5, seed=seed)
    if kind == "rrg3_pm":
        return I.random_regular3(12, coupling="pm1", seed=seed)
    if kind == "chimera1":
        inst = I.chimera(1, coupling="pm1", seed=seed)
        return inst
    if kind == "potts_gauss":
        return I.potts_square(2, 4, seed=seed)
    if kind == "potts_pm":
        return I.potts_square(3, 3, coupling="pm1", seed=seed)
    if kind == "cubic_pm":
        return I.cubic_lattice(2, 2, 3, coupling="pm1", seed=seed)
    if kind == "cubic_gauss_h":
        return I.cubic_lattice(2, 2, 3, coupling="gauss", field_sigma=0.5, seed=seed)
    if kind == "random_graph_int_h":
        n = 10
        pairs = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.35]
        e = np.asarray(pairs, np.int32).reshape(-1, 2)
        return dict(n=n, q=2, edges=e, J=rng.integers(-2, 3, len(e)).astype(np.float32),
                    h=rng.integers(-1, 2, n).astype(np.float32), name="rg", seed=seed)
    raise KeyError(kind)


KINDS = ["square_pm", "square_gauss_h", "rrg3_pm", "chimera1", "potts_gauss", "potts_pm",
         "cubic_pm", "cubic_gauss_h", "random_graph_int_h"]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("seed", range(4))
def test_elimination_matches_brute_force(kind, seed):
    inst = _random_small(kind, seed)
    b = O.brute_force(inst)
    rng = np.random.default_rng(100 + seed)
    orders = [None, list(range(inst["n"])), rng.permutation(inst["n"]).tolist()]
    for order in orders:
        s = O.solve(inst, order=order)
        assert s["E"] == pytest.approx(b["E"], rel=1e-12, abs=1e-12)
        assert s["count"] == b["count"]
        st = tuple(s["state"].tolist())
        assert st in set(map(tuple, b["states"].tolist()))


def test_first_index_tie_rule():
    # Two degenerate ground states (++ and --): the first-index rule of the
    # footnote in Sec. III keeps index 0 for the last-eliminated spin.
    inst = _inst_from_case(_cases()[0])
    s = O.solve(inst, order=[0, 1])
    assert s["state"].tolist() == [0, 0]


# ---------------------------------------------------------------- closed forms

GRAPHS = {
    "square8": lambda seed: I.square_lattice(8, coupling="gauss", seed=seed),
    "square5x9_pm": lambda seed: I.square_lattice(5, 9, coupling="pm1", seed=seed),
    "chimera2": lambda seed: I.chimera(2, coupling="gauss", seed=seed),
    "rrg3_24": lambda seed: I.random_regular3(24, coupling="gauss", seed=seed),
    "cubic4": lambda seed: I.cubic_lattice(4, coupling="gauss", seed=seed),
}


@pytest.mark.parametrize("g", list(GRAPHS))
def test_ferromagnet_closed_form(g):
    inst = I.ferromagnet(GRAPHS[g](7))
    s = O.solve(inst)
    exact = -float(np.sum(np.abs(inst["J"].astype(np.float64))))
    assert s["E"] == pytest.approx(exact, rel=1e-12)
    assert s["count"] == 2
    st = set(s["state"].tolist())
    assert len(st) == 1


@pytest.mark.parametrize("g", list(GRAPHS))
def test_mattis_planted_closed_form(g):
    inst, tau = I.planted(GRAPHS[g](3), seed=11)
    s = O.solve(inst)
    assert s["E"] == pytest.approx(-float(np.abs(inst["J"].astype(np.float64)).sum()), rel=1e-12)
    assert s["count"] == 2
    sig = 1 - 2 * s["state"].astype(np.int64)
    assert np.all(sig == tau) or np.all(sig == -tau)


def test_zero_coupling_fields_and_big_counts():
    # J = 0: E = -sum |h|, count 2^(number of h_i == 0), sigma_i = sign(h_i).
    inst = I.square_lattice(6, 7, coupling="zero", seed=1)
    rng = np.random.default_rng(5)
    h = rng.integers(-2, 3, inst["n"]).astype(np.float32)
    inst = dict(inst, h=h)
    s = O.solve(inst)
    assert s["E"] == -float(np.abs(h).sum())
    assert s["count"] == 2 ** int((h == 0).sum())
    nz = h != 0
    assert np.all((1 - 2 * s["state"][nz].astype(int)) == np.sign(h[nz]))


def test_zero_coupling_counts_beyond_int64():
    # 2^144 ground states: exercises the exact (Python-integer) count path.
    inst = I.square_lattice(12, coupling="zero", seed=0)
    s = O.solve(inst, order=I.square_sweep_order(12), config=False)
    assert s["E"] == 0.0
    assert s["count"] == 2 ** 144


def _ring(n, J):
    e = np.array([(i, (i + 1) % n) for i in range(n)], np.int32)
    return dict(n=n, q=2, edges=e, J=np.asarray(J, np.float32), h=None, name="ring", seed=0)


@pytest.mark.parametrize("n", [3, 4, 7, 12, 31])
def test_frustrated_ring_closed_form(n):
    rng = np.random.default_rng(n)
    for _ in range(3):
        J = np.where(rng.random(n) < 0.5, 1.0, -1.0)
        s = O.solve(_ring(n, J))
        if np.prod(J) > 0:
            assert (s["E"], s["count"]) == (-n, 2)
        else:
            assert (s["E"], s["count"]) == (-(n - 2), 2 * n)


def test_frustrated_ring_brute_force():
    for n in (5, 6):
        J = np.ones(n)
        J[2] = -1
        b = O.brute_force(_ring(n, J))
        assert (b["E"], b["count"]) == (-(n - 2), 2 * n)


@pytest.mark.parametrize("n", [2, 5, 9, 16])
def test_potts_colourings_path_and_cycle(n):
    # Antiferromagnetic Potts (J = -1): E = number of equal neighbours; with a
    # proper 3-colouring E = 0 and the degeneracy is the chromatic polynomial at 3.
    path = np.array([(i, i + 1) for i in range(n - 1)], np.int32).reshape(-1, 2)
    inst = dict(n=n, q=3, edges=path, J=-np.ones(len(path), np.float32), h=None, name="p", seed=0)
    s = O.solve(inst)
    assert (s["E"], s["count"]) == (0.0, 3 * 2 ** (n - 1))
    if n >= 3:
        cyc = np.array([(i, (i + 1) % n) for i in range(n)], np.int32)
        inst = dict(inst, edges=cyc, J=-np.ones(n, np.float32))
        s = O.solve(inst)
        assert (s["E"], s["count"]) == (0.0, 2 ** n + 2 * (-1) ** n)


def _tree_dp(inst, root=0):
    """Leaf-to-root max-sum on a tree, written from the definition (Sec. III)."""
    n = inst["n"]
    adj = [[] for _ in range(n)]
    for (u, v), j in zip(inst["edges"].tolist(), inst["J"].astype(float).tolist()):
        adj[u].append((v, j))
        adj[v].append((u, j))
    h = np.zeros(n) if inst["h"] is None else inst["h"].astype(float)
    sval = [1.0, -1.0]

    def up(v, parent):
        # best (value, count) of the subtree of v for each state of v
        best = [h[v] * sval[a] for a in range(2)]
        cnt = [1, 1]
        for w, j in adj[v]:
            if w == parent:
                continue
            bw, cw = up(w, v)
            for a in range(2):
                cand = [j * sval[a] * sval[b] + bw[b] for b in range(2)]
                m = max(cand)
                best[a] += m
                cnt[a] *= sum(cw[b] for b in range(2) if cand[b] == m)
        return best, cnt

    b, c = up(root, -1)
    m = max(b)
    return -m, sum(c[a] for a in range(2) if b[a] == m)


@pytest.mark.parametrize("seed", range(4))
def test_tree_graphs_match_max_sum(seed):
    rng = np.random.default_rng(seed)
    n = 40
    parent = [int(rng.integers(0, i)) for i in range(1, n)]
    e = np.array([(p, i + 1) for i, p in enumerate(parent)], np.int32)
    integral = seed % 2 == 0
    J = rng.integers(-2, 3, n - 1).astype(np.float32) if integral else \
        rng.standard_normal(n - 1).astype(np.float32)
    h = rng.integers(-1, 2, n).astype(np.float32) if integral else \
        (0.3 * rng.standard_normal(n)).astype(np.float32)
    inst = dict(n=n, q=2, edges=e, J=J, h=h, name="tree", seed=seed)
    E, cnt = _tree_dp(inst)
    s = O.solve(inst)
    assert s["E"] == pytest.approx(E, rel=1e-12, abs=1e-12)
    if integral:
        assert s["count"] == cnt


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(3))
def test_pm_j_parity_and_even_degeneracy(seed):
    inst = I.square_lattice(10, coupling="pm1", seed=seed)
    s = O.solve(inst, order=I.square_sweep_order(10))
    m = len(inst["edges"])
    assert int(s["E"]) == s["E"]
    assert (int(s["E"]) - m) % 2 == 0
    assert s["count"] % 2 == 0
    assert s["E"] >= -m
    assert O.energy(inst, s["state"]) == s["E"]
    s2 = O.solve(inst)                                  # min-fill order
    assert (s2["E"], s2["count"]) == (s["E"], s["count"])


@pytest.mark.parametrize("seed", range(3))
def test_potts_degeneracy_multiple_of_three(seed):
    inst = I.potts_square(4, 5, coupling="pm1", seed=seed)
    s = O.solve(inst)
    assert s["count"] % 3 == 0
    assert O.energy(inst, s["state"]) == s["E"]


def test_finite_difference_in_h_gives_configuration():
    # Sec. III: E_min is piecewise linear in h, dE/dh_i = -sigma_i.
    inst = I.square_lattice(4, 5, coupling="gauss", field_sigma=0.5, seed=3)
    s = O.solve(inst)
    sig = 1 - 2 * s["state"].astype(np.int64)
    eps = 1e-4
    for i in range(inst["n"]):
        hp = inst["h"].astype(np.float64).copy()
        hm = hp.copy()
        hp[i] += eps
        hm[i] -= eps
        Ep = O.solve(dict(inst, h=hp.astype(np.float32)), config=False, count=False)["E"]
        Em = O.solve(dict(inst, h=hm.astype(np.float32)), config=False, count=False)["E"]
        d = (Ep - Em) / (np.float32(hp[i]) - np.float32(hm[i]))
        assert d == pytest.approx(-sig[i], abs=1e-3)


# ---------------------------------------------------------------- semiring

def test_maxplus_matmul_is_best_path():
    rng = np.random.default_rng(0)
    dims = [3, 4, 2, 5]
    mats = [rng.integers(-5, 6, (dims[i], dims[i + 1])) for i in range(3)]
    C = S.maxplus_matmul(S.maxplus_matmul(mats[0], mats[1]), mats[2])
    for a in range(dims[0]):
        for d in range(dims[3]):
            paths = [mats[0][a, b] + mats[1][b, c] + mats[2][c, d]
                     for b in range(dims[1]) for c in range(dims[2])]
            assert C[a, d] == max(paths)
    ident = np.full((4, 4), -np.inf)
    np.fill_diagonal(ident, 0.0)
    A = rng.standard_normal((3, 4))
    assert np.array_equal(S.maxplus_matmul(A, ident), A)


def test_counting_matmul_counts_best_paths():
    rng = np.random.default_rng(1)
    dims = [2, 5, 4, 3]
    mats = [rng.integers(-1, 2, (dims[i], dims[i + 1])) for i in range(3)]
    ones = [np.ones_like(m) for m in mats]
    x, n = S.counting_matmul(mats[0], ones[0], mats[1], ones[1])
    x, n = S.counting_matmul(x, n, mats[2], ones[2])
    for a in range(dims[0]):
        for d in range(dims[3]):
            paths = [mats[0][a, b] + mats[1][b, c] + mats[2][c, d]
                     for b in range(dims[1]) for c in range(dims[2])]
            assert x[a, d] == max(paths)
            assert n[a, d] == paths.count(max(paths))
    p = (1 << 61) - 1
    big = np.full((1, 2), 1 << 60, dtype=object)
    bx = np.zeros((1, 2))
    x2, n2 = S.counting_matmul(bx, big, bx.T, big.T, mod=p)
    assert n2[0, 0] == (2 * (1 << 120)) % p


# ---------------------------------------------------------------- planted mistake

def test_planted_sign_mistake_is_caught(monkeypatch):
    """A wrong bond-tensor sign in the oracle must break a pin."""
    from oracle import elimination as E

    orig = E.local_tensors

    def wrong(inst, count=True):
        fs = orig(inst, count)
        for f in fs:
            if len(f.scope) == 2:
                f.val = -f.val
        return fs

    monkeypatch.setattr(E, "local_tensors", wrong)
    inst = _inst_from_case(_cases()[2])        # antiferromagnetic triangle
    s = E.solve(inst)
    assert (s["E"], s["count"]) != (-1.0, 6)


def test_potts_planted_colouring_is_ground_state():
    inst, tau = I.potts_planted(I.potts_square(3, 4, seed=2), seed=3)
    b = O.brute_force(inst)
    assert b["E"] == pytest.approx(-float(np.maximum(inst["J"].astype(np.float64), 0).sum()))
    assert tuple(tau.tolist()) in set(map(tuple, b["states"].tolist()))


def test_chimera_sweep_order_is_a_permutation_and_exact():
    for L in (1, 2, 3):
        seq = I.chimera_sweep_order(L)
        assert sorted(seq.tolist()) == list(range(8 * L * L))
    inst = I.chimera(2, coupling="pm1", seed=4)
    a = O.solve(inst, order=I.chimera_sweep_order(2))
    b = O.solve(inst)
    assert (a["E"], a["count"]) == (b["E"], b["count"])


def test_cubic_lattice_graph():
    """Open L x W x H cubic lattice: 3LWH - WH - LH - LW bonds, degree 6 inside."""
    e = I.cubic_edges(6)
    assert len(e) == 3 * 216 - 3 * 36 == 540
    assert len({tuple(sorted(x)) for x in e.tolist()}) == len(e)
    deg = np.bincount(e.ravel(), minlength=216)
    assert deg.max() == 6 and deg.min() == 3
    assert deg[(1 * 6 + 1) * 6 + 1] == 6 and deg[0] == 3
    assert len(I.cubic_edges(2, 3, 4)) == 3 * 24 - 12 - 8 - 6
