"""FP64 CPU oracle of the anisotropic ADE entropic lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
literal restatement of the method in double precision (PyTorch CPU tensor
ops, float64), written from the paper's Section 2 and the Strang-split source
of Section 3.3.  It exists to check the CUDA library, never to stand in for
it: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it.  It shares no code with the
CUDA path (``paper_2605_01774_gb300``) and imports nothing from it; the only
code both sides consume is the seeded input generator ``synth``.

Readings of passages where the paper is silent or ambiguous are listed in the
module docstring of :mod:`oracle.elbm` and in the design notes.

Pins (tests that fix this oracle against something other than itself) live in
``tests/test_oracle_*.py``.  Functions with no such pin say so in their
docstring ("parity unpinned").
"""
from .elbm import *  # noqa: F401,F403
