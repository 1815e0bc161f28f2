"""CPU oracle for the TCI contraction path (TEST INFRASTRUCTURE ONLY).

This package is the slow, plain, obviously-correct reference that the CUDA
library is checked against.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library and its
Python binding never do, and it shares no code with them (the only common
module is ``tci_synth``, which draws seeded inputs and holds no arithmetic of
the method).

All floating point is float64 / complex128.  Each function names the passage
of the TCI paper (arXiv 2512.23917) or the textbook definition it follows.

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: brute-force index sums, the paper's worked examples, exact
diagonalisation of Heisenberg chains, closed forms and invariants.  No
function here is "parity unpinned".
"""
from .contract import contract, contract_bruteforce, LabelError, UnsupportedLabels  # noqa: F401
from . import heff, lanczos, blocksparse, tebd, precision  # noqa: F401
