"""Counts with one 31-bit prime per pass (4-byte residue planes).

When the residue planes of n 61-bit primes do not fit in device memory,
tn_count runs the counting contraction once per 31-bit prime, with a single
plane, and reconstructs the count by CRT over the passes (plus a witness
pass).  TN_COUNT_PASSES forces that path; the counts must equal those of the
61-bit path and of the oracle, bit for bit.  The chimera of 8 x 8 cells
(Sec. IV, 512 spins) needs it: its 61-bit planes would take about 1 TB.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import instances as I
import oracle as O
import paper_2008_06888_gb300 as P

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_06888_gb300 import build
    build.build()


def _cases():
    yield "square10_pm", I.square_lattice(10, coupling="pm1", seed=3), dict(order="greedy", seed=1)
    yield "chimera4_pm_greedy", I.chimera(4, coupling="pm1", seed=2), dict(order="greedy", seed=2)
    yield "chimera5_pm_cellrow", I.chimera(5, coupling="pm1", seed=7), \
        dict(order="sweep", seq=I.chimera_sweep_order(5))
    yield "potts6_gauss", I.potts_square(6, coupling="gauss", seed=90), \
        dict(order="sweep", seq=I.square_sweep_order(6))
    yield "square7_pm_field", I.square_lattice(7, coupling="pm1", seed=5), dict(order="greedy", seed=3)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_counts_in_passes_match_oracle_and_61_bit_path(case, monkeypatch):
    name, inst, kw = case
    o = O.solve(inst, order=kw.get("seq"), config=False)
    sg = P.SpinGlass(inst, **kw)
    try:
        c61, _, E61 = sg.count(3)
        monkeypatch.setenv("TN_COUNT_PASSES", "1")
        c31, _, E31 = sg.count(3)
        assert c61 == c31 == o["count"], (c61, c31, o["count"])
        if inst["q"] == 2 and np.all(np.round(inst["J"]) == inst["J"]):
            assert E61 == E31 == o["E"]
        else:
            assert abs(E31 - o["E"]) <= 1e-5 * max(1.0, abs(o["E"])) and E31 == E61
    finally:
        sg.close()


def test_counts_in_passes_beyond_64_bits(monkeypatch):
    """J = 0 on an 8 x 8 lattice: every state is a ground state, 2^64 of them;
    two 61-bit primes (four 31-bit passes + witness) hold it exactly, one does
    not (the witness pass reports the overflow)."""
    inst = I.square_lattice(8, coupling="pm1", seed=0)
    inst = dict(inst, J=np.zeros_like(inst["J"]))
    sg = P.SpinGlass(inst, order="sweep", seq=I.square_sweep_order(8))
    try:
        monkeypatch.setenv("TN_COUNT_PASSES", "1")
        c, _, E = sg.count(2)
        assert E == 0.0 and c == 1 << 64
        from paper_2008_06888_gb300 import binding as B
        with pytest.raises(B.TNError) as e:
            sg.count(1)
        assert e.value.status == B.TN_EOVERFLOW
    finally:
        sg.close()


_CHIMERA8 = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import instances as I
import paper_2008_06888_gb300 as P
out = {}
inst, tau = I.planted(I.chimera(8, coupling="pm1", seed=3), seed=4)
sg = P.SpinGlass(inst, order="sweep", seq=I.chimera_sweep_order(8))
c, ln, E = sg.count(1)
out["planted"] = [E, str(c)]
sg.close()
inst = I.chimera(8, coupling="pm1", seed=8)
sg = P.SpinGlass(inst, order="sweep", seq=I.chimera_sweep_order(8))
E0 = sg.energy()
c, ln, E = sg.count(2)
out["random"] = [E0, E, str(c), ln / inst["n"]]
print(json.dumps(out))
"""


def test_chimera8_counts_in_passes():
    """Chimera 8 x 8 cells (512 spins, 1472 couplers) in cell-row order, peak 2^33
    elements: the 61-bit planes do not fit, so the count runs in 31-bit passes
    (one 4-byte plane, a 240 GB arena).  In a fresh process, for the device
    memory.  Mattis-planted: E = -1472 with exactly 2 ground states; a random
    +-J instance: the count's E equals tn_energy's, the count is even (global
    flip) and its entropy per spin is small and positive (the paper's ensemble
    value is about 0.03)."""
    r = subprocess.run([sys.executable, "-c", _CHIMERA8, ROOT], capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    E, c = out["planted"]
    assert E == -1472.0 and int(c) == 2
    E0, E, c, s = out["random"]
    assert E0 == E and int(c) >= 2 and int(c) % 2 == 0
    assert E >= -1472 and int(E) % 2 == 0     # +-J: E_min = n_edges (mod 2)
    assert 0.0 < s < 0.1


@pytest.mark.parametrize("case", list(_cases())[:4], ids=lambda c: c[0])
def test_31_and_61_bit_planes_give_the_same_counts(case, monkeypatch):
    """The default residue planes (ceil(61 n / 31) 31-bit primes, 4 bytes each) and
    the 61-bit ones (TN_COUNT_61) reconstruct the same integers as the oracle; five
    61-bit primes (beyond nine 31-bit planes) take the 61-bit form."""
    name, inst, kw = case
    o = O.solve(inst, order=kw.get("seq"), config=False)
    sg = P.SpinGlass(inst, **kw)
    try:
        c31, _, E31 = sg.count(3)
        c5, _, E5 = sg.count(5)
        monkeypatch.setenv("TN_COUNT_61", "1")
        c61, _, E61 = sg.count(3)
        assert c31 == c61 == c5 == o["count"] and E31 == E61 == E5
    finally:
        sg.close()


def test_count_batch_31_bit_planes_beyond_2_to_the_61(monkeypatch):
    """J = 0 on an 8 x 8 lattice, three coupling sets in one batch: 2^64 ground
    states each, beyond one 61-bit prime, exact with the default planes (six 31-bit
    primes and a witness)."""
    base = I.square_lattice(8, coupling="pm1", seed=0)
    sg = P.SpinGlass(dict(base, J=np.zeros_like(base["J"])), order="sweep",
                     seq=I.square_sweep_order(8))
    try:
        Jz = np.zeros((3, len(base["J"])), np.float32)
        E, counts, status = sg.count_batch(Jz, limbs_per=4)
        assert np.all(status == 0) and all(c == 1 << 64 for c in counts)
        assert np.all(E == 0.0)
    finally:
        sg.close()
