"""CPU oracle for the tropical tensor-network contraction -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package.  The CUDA library never imports, links or calls
it, and it shares no code with the library: the only common module is the
seeded instance generator (``instances``), which holds no contraction
arithmetic.

Everything here is plain numpy in float64 with exact Python-integer counts:

  energy.py       Eq. 1 (Ising) and the Potts energy, evaluated directly.
  brute.py        exhaustive enumeration of all q^N states (N <= ~20).
  elimination.py  tropical variable elimination (max-sum bucket elimination)
                  with counting tuples and an argmax traceback for sigma*.
  semiring.py     the element algebra of Eq. 2 and of the counting tuples, and
                  max-plus / counting matrix products written from their
                  definitions.

Pins (tests/test_oracle_pins.py) tie these to values fixed by the paper and by
mathematics: hand-derived golden examples, brute force, closed forms
(ferromagnet, Mattis-planted, J = 0, frustrated rings, proper 3-colourings),
tree max-sum, parity invariants and order independence.
"""
from .energy import energy, energies_of
from .brute import brute_force
from .elimination import solve, min_fill_order
from . import semiring

__all__ = ["energy", "energies_of", "brute_force", "solve", "min_fill_order", "semiring"]
