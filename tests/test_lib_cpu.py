"""Host-side checks of libtn.so that need no GPU: every symbol declared in
include/tn.h is exported, argument validation, and the planner (orders,
step classification, memory plan) reachable through the C ABI."""
import os
import re
import subprocess

import numpy as np
import pytest

import instances as I
import paper_2008_06888_gb300 as P
from paper_2008_06888_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tn.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_06888_gb300 import build
    build.build()


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", txt)))


def test_header_symbols_exported():
    names = declared()
    assert "tn_build" in names and "tn_count" in names and "tn_config" in names
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = B.lib()
    for n in names:
        assert hasattr(L, n)
    assert set(names) <= set(B._SIGS)


def test_build_rejects_bad_input():
    good = I.square_lattice(3, coupling="pm1", seed=0)
    bad = dict(good, edges=np.array([[0, 0]], np.int32), J=np.array([1.0], np.float32))
    with pytest.raises(B.TNError) as e:
        B.tn_build(bad)
    assert e.value.status == B.TN_EINVAL
    dup = dict(good, edges=np.array([[0, 1], [1, 0]], np.int32), J=np.ones(2, np.float32))
    with pytest.raises(B.TNError):
        B.tn_build(dup)
    with pytest.raises(B.TNError):
        B.tn_build(dict(good, q=4))
    with pytest.raises(B.TNError):
        B.tn_build(dict(I.potts_square(2, seed=0), h=np.zeros(4, np.float32)))
    with pytest.raises(B.TNError):
        B.tn_build(dict(good, J=np.full(len(good["J"]), 0.5, np.float32)), dtype=B.TN_DTYPE_I32)


def test_compute_before_order_is_state_error():
    c = B.tn_build(I.square_lattice(3, coupling="pm1", seed=0))
    try:
        with pytest.raises(B.TNError) as e:
            B.tn_backward(c, 9)
        assert e.value.status in (B.TN_ESTATE, B.TN_ECUDA)
    finally:
        B.tn_destroy(c)


def test_sweep_order_width():
    # row-by-row elimination of an L x L lattice keeps about L+1 spins live
    for L in (4, 6, 10):
        sg = P.SpinGlass(I.square_lattice(L, coupling="pm1", seed=1), order="sweep",
                         seq=I.square_sweep_order(L))
        assert L - 1 <= sg.log2_peak <= L + 1
        info = sg.plan_info()
        assert info["n_steps"] >= 2 * L * (L - 1) - 1
        assert info["n_transposes"] == 0


def test_greedy_order_is_deterministic_and_valid():
    inst = I.random_regular3(40, coupling="gauss", seed=4)
    a = P.SpinGlass(inst, order="greedy", seed=7, restarts=8)
    b = P.SpinGlass(inst, order="greedy", seed=7, restarts=8)
    assert (a.log2_peak, a.log2_ops) == (b.log2_peak, b.log2_ops)
    assert a.log2_peak < 20


def test_greedy_beats_plain_sweep_on_24x24():
    inst = I.square_lattice(24, coupling="gauss", field_sigma=0.1, seed=1)
    g = P.SpinGlass(inst, order="greedy", seed=1, restarts=32)
    s = P.SpinGlass(inst, order="sweep", seq=I.square_sweep_order(24))
    assert g.log2_peak <= 25 and g.log2_ops < s.log2_ops


def test_explicit_tree_order():
    inst = I.square_lattice(2, coupling="pm1", seed=0)   # 4 bonds, leaves 0..3
    c = B.tn_build(inst)
    try:
        assert B.tn_leaf_count(c) == 4
        pk, ops = B.tn_order(c, B.TN_ORDER_TREE, [0, 1, 2, 3, 4, 5])
        assert pk <= 3
        with pytest.raises(B.TNError):
            B.tn_order(c, B.TN_ORDER_TREE, [0, 1, 0, 2])        # tensor used twice
        with pytest.raises(B.TNError):
            B.tn_order(c, B.TN_ORDER_TREE, [0, 1])              # does not reach a root
    finally:
        B.tn_destroy(c)


def test_isolated_and_leaf_spins_plan():
    inst = dict(n=5, q=2, edges=np.array([[0, 1], [1, 2]], np.int32),
                J=np.array([1, -1], np.float32), h=np.array([0, 1, 0, 2, 0], np.float32),
                name="t", seed=0)
    sg = P.SpinGlass(inst, order="greedy")
    assert sg.plan_info()["n_steps"] >= 3


def _is_prime(n):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):   # deterministic below 3.3e24
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def test_count_primes_are_61_bit_primes():
    src = open(os.path.join(ROOT, "paper_2008_06888_gb300", "csrc", "api.cpp")).read()
    m = re.search(r"kPrimeC\[TN_MAX_PRIMES\]\s*=\s*\{([^}]*)\}", src)
    cs = [int(x) for x in m.group(1).split(",")]
    assert len(set(cs)) == len(cs) == 9
    for c in cs:
        p = (1 << 61) - c
        assert _is_prime(p) and c < 1024


def test_pass_primes_are_31_bit_primes():
    """The one-prime-per-pass counts use 2^31 - c primes with c < 1024 (the
    device reduction folds the 62-bit product twice, which needs c < 2^10)."""
    src = open(os.path.join(ROOT, "paper_2008_06888_gb300", "csrc", "api.cpp")).read()
    m = re.search(r"kPrime31C\[kPasses31Max\]\s*=\s*\{([^}]*)\}", src)
    cs = [int(x) for x in m.group(1).split(",")]
    assert len(set(cs)) == len(cs) == 17
    for c in cs:
        assert _is_prime((1 << 31) - c) and c < 1024
    # enough passes for 8 61-bit primes plus a witness
    assert (61 * 8 + 30) // 31 + 1 <= len(cs)


def test_no_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    sg = P.SpinGlass(I.square_lattice(3, coupling="pm1", seed=0))
    with pytest.raises(B.TNError) as e:
        sg.energy()
    assert e.value.status == B.TN_ECUDA


@pytest.mark.parametrize("seed", range(4))
def test_max2sat_couplings_reproduce_the_clause_cost(seed):
    """cost(x) = (E_ising(sigma) + n_clauses) / 4 for every assignment, x true <-> sigma = +1
    (E_ising by Eq. 1 in the oracle, cost from the clauses by the oracle)."""
    import oracle
    from oracle import max2sat as M
    sat = I.max2sat_regular3(12, seed=seed)
    if seed == 3:        # clauses repeated on one pair are merged into one edge
        extra = np.array([[1, -2], [-1, -2]], np.int32)
        sat = dict(sat, clauses=np.concatenate([sat["clauses"], extra]))
    e, J, h = B.tn_max2sat_couplings(sat)
    assert np.all(J == np.round(J)) and np.all(h == np.round(h))
    inst = dict(n=sat["n"], q=2, edges=e, J=J, h=h)
    idx = np.arange(1 << sat["n"])
    x = (idx[:, None] >> np.arange(sat["n"])[None, :]) & 1
    E = oracle.energies_of(inst, (1 - x).astype(np.int8))
    assert np.array_equal((E + len(sat["clauses"])) / 4, M.cost(sat, x))


def test_max2sat_rejects_bad_clauses():
    for lits in ([[1, 1]], [[0, 2]], [[1, 9]], [[-3, 3]]):
        with pytest.raises(B.TNError) as e:
            B.tn_build_max2sat(dict(n=4, clauses=np.array(lits, np.int32)))
        assert e.value.status == B.TN_EINVAL
    c = B.tn_build_max2sat(I.max2sat_regular3(10, seed=0))
    B.tn_order(c, B.TN_ORDER_GREEDY, None, 1, 4)
    B.tn_destroy(c)


def test_cubic_6x6x6_greedy_order_fits():
    c = B.tn_build(I.cubic_lattice(6, coupling="gauss", seed=1))
    pk, ops = B.tn_order(c, B.TN_ORDER_GREEDY, None, 1, 256)
    assert pk <= 31 and ops < 39
    B.tn_destroy(c)


def test_sample_argument_checks_before_any_device_work():
    g = B.tn_build(I.square_lattice(3, coupling="gauss", seed=1))
    with pytest.raises(B.TNError) as e:
        B.tn_sample(g, 9, 2)
    assert e.value.status == B.TN_ESTATE          # no order yet
    B.tn_order(g, B.TN_ORDER_GREEDY, None, 1, 4)
    with pytest.raises(B.TNError) as e:
        B.tn_sample(g, 9, 2)
    assert e.value.status == B.TN_EINVAL          # float couplings: no exact ties
    B.tn_destroy(g)
    c = B.tn_build(I.square_lattice(3, coupling="pm1", seed=1))
    B.tn_order(c, B.TN_ORDER_GREEDY, None, 1, 4)
    with pytest.raises(B.TNError) as e:
        B.tn_sample(c, 9, 2, order=[0, 1, 2, 3, 4, 5, 6, 7, 7])
    assert e.value.status == B.TN_EINVAL          # not a permutation
    B.tn_destroy(c)
    p = B.tn_build(I.potts_square(2, coupling="pm1", seed=1))
    B.tn_order(p, B.TN_ORDER_GREEDY, None, 1, 4)
    with pytest.raises(B.TNError) as e:
        B.tn_sample(p, 4, 2)
    assert e.value.status == B.TN_EINVAL          # Ising only
    B.tn_destroy(p)


def test_plan_launches_of_the_kernel_mix_case():
    """The chimera 4x4 greedy plan the GPU kernel-mix test runs has transposes,
    GEMMs and (in count mode) twice as many GEMM launches (values + residues)."""
    import instances as I
    inst = I.chimera(4, coupling="pm1", seed=2)
    c = B.tn_build(inst)
    try:
        B.tn_order(c, B.TN_ORDER_GREEDY, None, 2, 16)
        e = B.tn_plan_launches(c, "energy")
        n = B.tn_plan_launches(c, "count")
        assert e["transpose"] > 0 and e["gemm"] > 0
        assert n["gemm"] == 2 * e["gemm"] and n["transpose"] == 2 * e["transpose"]
        assert e["leaves"] == 1 and e["trace"] == 0
        assert B.tn_plan_launches(c, "config")["trace"] > 0
    finally:
        B.tn_destroy(c)
