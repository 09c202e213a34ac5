"""Counting register chains with vector accesses.

Where register legs of a counting chain (three legs, value + seven 4-byte
residue planes per element) sit at memory positions 0 and 1, the launcher
renumbers them to lead, and the kernel moves the 2 or 4 states that differ in
them with one 8- or 16-byte access per array.  TN_RCC_NO_VEC=1 keeps one
4-byte access per state.  Counts and energies must be identical either way and
equal the oracle's (Sec. II counting tuples).
"""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2008_06888_gb300 as P

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_DUMP = r"""
import sys
sys.path.insert(0, {root!r})
import instances as I
import paper_2008_06888_gb300 as P
from paper_2008_06888_gb300 import binding as B
inst = I.square_lattice({L}, coupling="pm1", seed={seed})
sg = P.SpinGlass(inst, order="sweep", seq=I.square_sweep_order({L}))
B.tn_plan_launches(sg.ctx, "count")
"""


def _low_leg_chains(L, seed):
    """Counting chains of the lowered count program with a register leg at
    memory position 0 (from the program dump; host only)."""
    env = dict(os.environ, TN_DUMP_PROGRAM="c")
    r = subprocess.run([sys.executable, "-c", _DUMP.format(root=ROOT, L=L, seed=seed)],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    n = 0
    for line in r.stderr.splitlines():
        m = re.search(r"chain mode 1 outer \d+ t 3 rin ([-\d ]+?) rout", line)
        if m and 0 in [int(x) for x in m.group(1).split()]:
            n += 1
    return n


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_06888_gb300 import build
    build.build()


@pytest.mark.parametrize("L,seed", [(11, 4), (12, 8)])
def test_vector_counting_chains_match_scalar_and_oracle(L, seed, monkeypatch):
    assert _low_leg_chains(L, seed) > 0   # the vector form is on this path
    inst = I.square_lattice(L, coupling="pm1", seed=seed)
    seq = I.square_sweep_order(L)
    o = O.solve(inst, order=seq, config=False)
    sg = P.SpinGlass(inst, order="sweep", seq=seq)
    try:
        c_vec, _, E_vec = sg.count(3)
    finally:
        sg.close()
    monkeypatch.setenv("TN_RCC_NO_VEC", "1")
    sg = P.SpinGlass(inst, order="sweep", seq=seq)
    try:
        c_sc, _, E_sc = sg.count(3)
    finally:
        sg.close()
    assert c_vec == c_sc == o["count"], (c_vec, c_sc, o["count"])
    assert E_vec == E_sc == o["E"]


def test_vector_counting_chains_in_a_mixed_batch(monkeypatch):
    """A small mixed batch through tn_batch_run: identical limbs with and
    without the vector form."""
    from paper_2008_06888_gb300 import binding as B
    insts = I.mixed_square_batch(24, Lmin=8, Lmax=14, seed=77)

    def run():
        sgs = [P.SpinGlass(x, order="sweep", seq=I.square_sweep_order(int(np.sqrt(x["n"]))))
               for x in insts]
        try:
            st, E, counts, status = B.tn_batch_run([s.ctx for s in sgs])
            return st, np.asarray(E).copy(), counts, np.asarray(status).copy()
        finally:
            for s in sgs:
                s.close()

    st1, E1, c1, s1 = run()
    monkeypatch.setenv("TN_RCC_NO_VEC", "1")
    st2, E2, c2, s2 = run()
    assert st1 == st2 == 0 and (s1 == 0).all() and (s2 == 0).all()
    assert np.array_equal(E1, E2) and c1 == c2


_DUMP_CHIMERA = r"""
import sys
sys.path.insert(0, {root!r})
import instances as I
import paper_2008_06888_gb300 as P
from paper_2008_06888_gb300 import binding as B
inst = I.chimera({L}, coupling="pm1", seed={seed})
sg = P.SpinGlass(inst, order="sweep", seq=I.chimera_sweep_order({L}))
B.tn_plan_launches(sg.ctx, "count")
"""


def _contiguous_16_state_gates(L, seed):
    """Gate steps of the count program with 16 new states stored as 16
    consecutive words per outer index (host only, from the program dump)."""
    env = dict(os.environ, TN_DUMP_PROGRAM="c")
    r = subprocess.run([sys.executable, "-c", _DUMP_CHIMERA.format(root=ROOT, L=L, seed=seed)],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    want = " nC " + " ".join(str(n) for n in range(16))
    return sum(1 for line in r.stderr.splitlines()
               if " Ks 2 Ns 16 " in line and line.rstrip().endswith(want))


@pytest.mark.parametrize("L,seed", [(4, 2), (5, 7)])
def test_vector_stores_of_16_state_counting_gates(L, seed, monkeypatch):
    """Counting gates with two contraction states and 16 new states (the
    chimera cell gates, Sec. IV) store four outputs per 16-byte access where
    the 16 outputs of an outer index are consecutive; TN_GATE_TC_NO_VEC=1
    stores them one by one.  Both equal the oracle."""
    assert _contiguous_16_state_gates(L, seed) > 0
    inst = I.chimera(L, coupling="pm1", seed=seed)
    seq = I.chimera_sweep_order(L)
    o = O.solve(inst, order=seq, config=False)
    res = []
    for novec in (False, True):
        if novec:
            monkeypatch.setenv("TN_GATE_TC_NO_VEC", "1")
        sg = P.SpinGlass(inst, order="sweep", seq=seq)
        try:
            c, _, E = sg.count(3)
        finally:
            sg.close()
        res.append((c, E))
    assert res[0] == res[1] == (o["count"], o["E"]), (res, o["count"], o["E"])
