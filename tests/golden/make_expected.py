"""Write tests/golden/expected_full.json from the CPU oracle only.

Full-size workloads whose oracle run takes minutes are solved once here and
stored with the sha256 digest of their input, so GPU tests can compare
against them in seconds.  Run from the repository root:

    python tests/golden/make_expected.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import instances as I  # noqa: E402
import oracle as O  # noqa: E402
from oracle import max2sat as M  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expected_full.json")

# indices into mixed_square_batch(2048, 8, 20, seed=2026): L = 10, 11, ..., 20, then three more L = 18
MIXED_2026 = [1, 19, 4, 33, 5, 26, 3, 12, 10, 0, 21, 11, 31, 46]
MIXED_BATCH_2026 = None


def cases():
    # 24x24 open square lattice, J ~ N(0,1), h ~ N(0, 0.1^2), float32 values
    yield "square24_gauss_h", I.square_lattice(24, coupling="gauss", field_sigma=0.1, seed=2008), \
        dict(order=I.square_sweep_order(24), count=False, config=True)
    # 16x16 +-J lattice with its exact degeneracy
    yield "square16_pm", I.square_lattice(16, coupling="pm1", seed=2008), \
        dict(order=I.square_sweep_order(16), count=True, config=True)
    # 12x12 3-state Potts glass, Gaussian couplings
    yield "potts12_gauss", I.potts_square(12, coupling="gauss", seed=2008), \
        dict(order=I.square_sweep_order(12), count=True, config=True)
    # 5x5x5 open cubic +-J lattice with its exact degeneracy
    yield "cubic5_pm", I.cubic_lattice(5, coupling="pm1", seed=2008), \
        dict(count=True, config=True)
    # Max-2-SAT on a random 3-regular graph, 140 variables (clause-tensor oracle)
    yield "max2sat140", I.max2sat_regular3(140, seed=2008), dict(count=True, config=True)
    # a second 5x5x5 +-J cubic lattice (batched cubic counts)
    yield "cubic5_pm_2009", I.cubic_lattice(5, coupling="pm1", seed=2009), \
        dict(count=True, config=False)
    # members of the 2048-instance mixed +-J batch (L uniform in 8..20, base seed 2026):
    # one instance of every L in 10..20, and three more with L = 18 (one batched plan)
    for k in MIXED_2026:
        inst = MIXED_BATCH_2026[k]
        L = int(round(inst["n"] ** 0.5))
        yield f"mixed2026_{k}", inst, dict(order=I.square_sweep_order(L), count=True,
                                           config=False)


def main():
    global MIXED_BATCH_2026
    MIXED_BATCH_2026 = I.mixed_square_batch(2048, Lmin=8, Lmax=20, seed=2026)
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    only = set(sys.argv[1:])
    for name, inst, kw in cases():
        if only and name not in only:
            continue
        t = time.time()
        r = M.solve(inst, **kw) if "clauses" in inst else O.solve(inst, **kw)
        out[name] = dict(
            name=inst["name"], seed=inst["seed"], digest=I.instance_digest(inst),
            E=r["E"], count=None if r["count"] is None else str(r["count"]),
            state="".join(str(int(x)) for x in r["state"]) if r["state"] is not None else None,
            oracle_seconds=round(time.time() - t, 1))
        print(name, out[name]["E"], out[name]["count"], out[name]["oracle_seconds"], flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
