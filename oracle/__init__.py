"""Plain FP64 CPU oracle of the MWU positive-LP solver (arXiv 2307.03307).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline legs, never by the library.  It shares no code
with the CUDA path; the two meet only at the seeded inputs of ``graphgen``.
"""
from . import lp, mwu, exact  # noqa: F401
