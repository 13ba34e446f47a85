"""CPU ORACLE -- test infrastructure, not part of the product.

A plain, slow, obviously-correct FP64 CPU implementation of what the SuperDC
conquering stage computes (Ou & Xia, arXiv 2108.04209).  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA library
in ``paper_2108_04209_gb300``; the two meet only through the seeded inputs of
``paper_2108_04209_gb300.inputs``.

Modules
  * ``rank1.c``   -- deflation (Remark 4.1), shifted secular roots
                    (Section 4.2, eqs. (4.13), (4.14), (4.17); stopping test eq. (4.12)),
                    Loewner zhat (eq. (4.23)), b (eq. (4.27)), Cauchy-like factor
                    application (eqs. (4.26), (4.29)), dense cyclic Jacobi;
  * ``rank1.py``  -- one complete rank-one step with its factor object;
  * ``superdc.py``-- Algorithm 1 (dividing), Algorithm 3 (conquering),
                    Algorithm 4 (superdcmv);
  * ``dense.py``  -- dense assembly of an HSS matrix and the accuracy metrics
                    gamma, delta, theta of Section 5.

Pins (tests/test_oracle_*.py): mpmath at 50 digits, closed forms (m = 1, 2,
z = e_k, the tridiagonal spectrum 3 - 2cos(k pi/(n+1))), numpy eigh, brute
force dense Jacobi, invariants (trace, Frobenius norm, interlacing,
orthogonality).
"""
from . import _build  # noqa: F401  (compiles rank1.c on first import)
