"""GPU parity on the 3D cubic lattice (Sec. IV) and on Max-2-SAT (App. D),
through the C ABI against the CPU oracle.  Integer energies, violated-clause
counts and every count of optimal states must match bit-exactly; float32
energies within 1e-5 relative."""
import numpy as np
import pytest

import instances as I
import oracle as O
from oracle import max2sat as M
import paper_2008_06888_gb300 as P
from paper_2008_06888_gb300 import binding as B

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_06888_gb300 import build
    build.build()


def close(a, b):
    return abs(a - b) <= REL * max(1.0, abs(b))


def state_of(sg):
    sigma, E = sg.config()
    return P.SpinGlass.state_indices(sigma, 2), E


# ------------------------------------------------------------ cubic lattice

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cubic4_pm_energy_count_state(seed):
    inst = I.cubic_lattice(4, coupling="pm1", seed=seed)
    o = O.solve(inst)
    sg = P.SpinGlass(inst, order="greedy", seed=seed, restarts=64)
    c, ln, E = sg.count(3)
    assert (E, c) == (o["E"], o["count"])
    st, E2 = state_of(sg)
    assert E2 == o["E"] and O.energy(inst, st) == o["E"]


def test_cubic4x4x5_gauss_fields_unique_state():
    inst = I.cubic_lattice(4, 4, 5, coupling="gauss", field_sigma=0.3, seed=7)
    o = O.solve(inst)
    assert o["count"] == 1
    sg = P.SpinGlass(inst, order="greedy", seed=2, restarts=64)
    st, E = state_of(sg)
    assert close(E, o["E"])
    assert np.array_equal(st, o["state"])


def test_cubic6_planted_pm_counts():
    inst, tau = I.planted(I.cubic_lattice(6, coupling="pm1", seed=5), seed=6)
    sg = P.SpinGlass(inst, order="greedy", seed=1, restarts=256)
    c, ln, E = sg.count(3)
    assert E == -540.0 and c == 2
    st, E2 = state_of(sg)
    sig = 1 - 2 * st.astype(np.int64)
    assert np.all(sig == tau) or np.all(sig == -tau)


def test_cubic6_gauss_two_orders_agree():
    inst = I.cubic_lattice(6, coupling="gauss", seed=11)
    res = []
    for seed in (1, 2):
        sg = P.SpinGlass(inst, order="greedy", seed=seed, restarts=256)
        st, E = state_of(sg)
        assert close(O.energy(inst, st), E)
        res.append((E, st))
        sg.close()
    assert close(res[0][0], res[1][0])
    # h = 0: the ground state is unique up to the global flip
    a, b = res[0][1].astype(np.int64), res[1][1].astype(np.int64)
    assert np.array_equal(a ^ a[0], b ^ b[0])


def test_cubic6_gauss_batch_matches_single():
    base = I.cubic_lattice(6, coupling="gauss", seed=1)
    sg = P.SpinGlass(base, order="greedy", seed=1, restarts=256)
    Js = np.stack([I.cubic_lattice(6, coupling="gauss", seed=40 + k)["J"] for k in range(2)])
    E, sig = sg.config_batch(Js, None)
    for k in range(2):
        sg.set_couplings(Js[k], None)
        s1, E1 = sg.config()
        assert E1 == E[k]
        assert np.array_equal(np.asarray(s1), np.asarray(sig[k]))


# ------------------------------------------------------------ Max-2-SAT

@pytest.mark.parametrize("N,seed", [(20, 5), (40, 1), (60, 2), (100, 3)])
def test_max2sat_vs_oracle(N, seed):
    sat = I.max2sat_regular3(N, seed=seed)
    o = M.solve(sat)
    ms = P.Max2SAT(sat, order="greedy", seed=seed, restarts=64)
    c, ln, E = ms.count(3)
    assert (E, c) == (o["E"], o["count"])
    assert ms.energy() == o["E"]
    x, E2 = ms.assignment()
    assert E2 == o["E"] and M.cost(sat, x)[0] == o["E"]


def test_max2sat_sign_patterns_batched():
    sat0 = I.max2sat_regular3(48, seed=8)
    rng = np.random.default_rng(3)
    sats = [dict(sat0, clauses=np.where(rng.integers(0, 2, sat0["clauses"].shape) == 1,
                                        -np.abs(sat0["clauses"]), np.abs(sat0["clauses"])
                                        ).astype(np.int32)) for _ in range(6)]
    ms = P.Max2SAT(sats[0], order="greedy", seed=1, restarts=64)
    cp = [P.Max2SAT.couplings(x) for x in sats]
    for c in cp[1:]:
        assert np.array_equal(c[0], cp[0][0])
    J = np.stack([c[1] for c in cp])
    h = np.stack([c[2] for c in cp])
    E, counts, status = ms.count_batch(J, h, 3)
    assert np.all(status == 0)
    for k, s in enumerate(sats):
        o = M.solve(s)
        assert (E[k], counts[k]) == (o["E"], o["count"]), k


def test_max2sat_batch_run_and_planted():
    sats = [I.max2sat_regular3(30 + 2 * k, seed=k) for k in range(5)]
    sats.append(I.max2sat_planted(I.max2sat_regular3(40, seed=9), seed=1)[0])
    objs = [P.Max2SAT(s, order="greedy", seed=1, restarts=16) for s in sats]
    st, E, counts, status = B.tn_batch_run([o.ctx for o in objs])
    assert st == 0 and np.all(status == 0)
    for k, s in enumerate(sats):
        o = M.solve(s)
        assert (E[k], counts[k]) == (o["E"], o["count"])
    assert E[-1] == 0


def test_max2sat_planted_n200_satisfied():
    sat, tau = I.max2sat_planted(I.max2sat_regular3(200, seed=4), seed=2)
    ms = P.Max2SAT(sat, order="greedy", seed=1, restarts=1024)
    x, cost = ms.assignment()
    assert cost == 0 and M.cost(sat, x)[0] == 0
    assert M.cost(sat, tau)[0] == 0


def test_max2sat_refuses_gradient():
    ms = P.Max2SAT(I.max2sat_regular3(20, seed=1), order="greedy", seed=1, restarts=4)
    ms.config()
    with pytest.raises(B.TNError) as e:
        ms.gradient()
    assert e.value.status == B.TN_ESTATE


@pytest.mark.parametrize("kind", ["sat", "square_pm"])
def test_streaming_count_gates_match_generic(kind, monkeypatch):
    """Counting gate steps in the streaming q = 2 form (k_gate2c) give the same
    energies and counts as the generic gate kernel (TN_NO_GATE2)."""
    def run():
        if kind == "sat":
            sat = I.max2sat_regular3(120, seed=6)
            o = P.Max2SAT(sat, order="greedy", seed=2, restarts=64)
        else:
            o = P.SpinGlass(I.square_lattice(14, coupling="pm1", seed=3), order="greedy",
                            seed=2, restarts=64)
        c, ln, E = o.count(3)
        o.close()
        return E, c
    a = run()
    monkeypatch.setenv("TN_NO_GATE2", "1")
    b = run()
    assert a == b


# ------------------------------------------------------------ ground-state sampling

def _degenerate_square(min_gs=6, max_gs=40):
    for seed in range(1, 200):
        inst = I.square_lattice(4, coupling="pm1", seed=seed)
        b = O.brute_force(inst)
        if min_gs <= b["count"] <= max_gs:
            return inst, b
    raise RuntimeError("no degenerate instance found")


def test_sample_draws_every_ground_state_uniformly():
    """Sec. III: spins fixed one at a time with their conditional probabilities
    (exact count ratios) give uniform samples of the ground states."""
    inst, b = _degenerate_square()
    sg = P.SpinGlass(inst, order="greedy", seed=1, restarts=16)
    S = 40 * b["count"]
    sig = sg.sample(S, seed=7)
    gs = {tuple(x) for x in b["states"].tolist()}
    freq = {}
    for row in sig:
        st = tuple(((1 - row.astype(np.int64)) // 2).tolist())
        assert st in gs
        freq[st] = freq.get(st, 0) + 1
    assert len(freq) == len(gs)
    expct = S / len(gs)
    chi2 = sum((freq[g] - expct) ** 2 / expct for g in gs)
    dof = len(gs) - 1
    assert chi2 <= dof + 6 * np.sqrt(2 * dof) + 1, (chi2, dof)
    # the same seed gives the same samples, another order still ground states
    assert np.array_equal(sg.sample(S, seed=7)[:10], sig[:10])
    other = sg.sample(20, seed=8, order=np.arange(inst["n"])[::-1])
    for row in other:
        assert O.energy(inst, ((1 - row.astype(np.int64)) // 2).astype(np.int8)) == b["E"]


def test_sample_max2sat_optimal_assignments():
    sat = I.max2sat_regular3(18, seed=2)
    o = M.brute_force(sat)
    ms = P.Max2SAT(sat, order="greedy", seed=1, restarts=16)
    sig = ms.sample(30, seed=3)
    xs = {tuple((row > 0).astype(int).tolist()) for row in sig}
    for x in xs:
        assert M.cost(sat, np.array(x))[0] == o["E"]
    assert len(xs) > 1 if o["count"] > 1 else len(xs) == 1


# ------------------------------------------------------------ stored oracle values (larger sizes)

def _expected(name):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "expected_full.json")
    with open(path) as f:
        d = json.load(f)
    if name not in d:
        pytest.skip(f"{name} not in expected_full.json")
    return d[name]


def test_full_cubic5_pm_counts():
    exp = _expected("cubic5_pm")
    inst = I.cubic_lattice(5, coupling="pm1", seed=2008)
    assert I.instance_digest(inst) == exp["digest"]
    sg = P.SpinGlass(inst, order="greedy", seed=1, restarts=64)
    c, _, E = sg.count(3)
    assert E == exp["E"] and c == int(exp["count"])
    st, E2 = state_of(sg)
    assert E2 == E and O.energy(inst, st) == E


def test_full_max2sat140_counts():
    exp = _expected("max2sat140")
    sat = I.max2sat_regular3(140, seed=2008)
    assert I.instance_digest(sat) == exp["digest"]
    ms = P.Max2SAT(sat, order="greedy", seed=1, restarts=64)
    c, _, E = ms.count(3)
    assert E == exp["E"] and c == int(exp["count"])
    x, E2 = ms.assignment()
    assert E2 == E and M.cost(sat, x)[0] == E
