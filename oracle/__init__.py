"""CPU oracle for the tensor-network PTSBE hot path (arxiv 2604.08467).

TEST INFRASTRUCTURE ONLY.  Plain, slow, complex128 NumPy code that states what
the GPU path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
library under ``paper_2604_08467_gb300`` never does, and this package never
imports that library.  The two share only the seeded input generators in
``workloads``.

Modules:

* ``philox``      counter-based Philox4x32-10 generator (Salmon et al., SC'11)
* ``pts``         pre-trajectory sampling of Kraus error sets (Sec. II-C) and the
                  unified-path-variation tensor merge (Sec. III-A)
* ``statevector`` per-trajectory state vectors and block marginals (Sec. II-B)
* ``mps``         exact matrix-product-state contraction for 1D circuits, an
                  independent second method for large qubit counts
* ``densmat``     exact density-matrix evolution (Sec. I / II-A)
* ``sampling``    exact-integer CDF sampling and proportional non-degenerate
                  batched sampling (Sec. III-B)
"""
