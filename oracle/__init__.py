"""FP64 CPU oracle of the SPH step (NL, PI, SU) and of its gradient.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call or execute anything here.  The
oracle shares no code with the CUDA library (``paper_1110_3711_gb300``) and
neither imports the other; the seeded inputs both consume come from
``sphcases``.

Parity status of each function is listed in the header of ``sph_oracle.c`` and
pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
