"""CPU oracle for the compressed H-matrix-vector product (Kriemann, "Hierarchical Lowrank
Arithmetic with Binary Compression").

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct FP64 restatement of
what the GPU path computes. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may import it. It shares no code with the product
package (``paper_2308_10960_gb300``); its only shared dependency is the seeded input module
``synth`` (problem definition, no method arithmetic).

Modules
-------
formats  : unit roundoff and dynamic range of IEEE-754 style formats (Table 1, Table 2).
afl      : the AFL encoder/decoder (Section 3.2, with the remark on scaling by 1/m_min and
           shifting by 1) and the APLR per-column precision rule (Section 3.3).
hmatrix  : cluster tree (Def. 2.1), block tree with standard admissibility (Def. 2.2,
           Section 5.1), H-matrix with eps-accurate lowrank leaves (Def. 2.3, Eq. 1), lowrank
           approximation by truncated SVD or ACA followed by SVD recompression (Algorithm 1),
           and compression of every leaf (dense: AFL at eps; lowrank: AFL-APLR).
matvec   : y_out = y_in + A~ x with compensated summation (Section 5.4), dense products.
cg       : unpreconditioned conjugate gradients on the decoded operator.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` (closed forms,
Table 1/2, hand-worked codes, library SVD, brute-force dense products, invariants).
"""
