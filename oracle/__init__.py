"""CPU oracle of the Ozaki-II scheme (arXiv 2602.02549).

TEST INFRASTRUCTURE ONLY: only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call, link or execute anything
in this package.  It shares no code with the GPU library.

Pinning (see tests/test_oracle_*.py): exact rationals on tiny inputs, integer
inputs that must come out exact, the CRT round trip (Theorem 1), Lemmas 0-4 and
the bound of Theorem 2 on every case; the bound evaluators themselves (bounds,
bound_from_exponents, bound_splitk, mu_band) against the same formulas evaluated
in exact rational arithmetic, with planted mistakes.  Parity unpinned: the
bound-chosen N rules (normwise and componentwise) and the fast-mode scaling are
readings, not results printed in the paper.

Modules: ozaki2 (Algorithms 1-3, bounds, N rules), constants (exact tables),
sharded (row-sharded Algorithms 1-3 over torch.distributed ranks), moduli (per-N
moduli tables).
"""
