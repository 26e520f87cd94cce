"""Plain FP64 CPU oracle for randomized compression of rank-structured matrices.

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``; the product path (``paper_1503_07152_gb300``) never
imports, links or executes anything in here, and nothing here imports the
product.  It is deliberately slow and obviously correct: NumPy FP64, LAPACK
(through NumPy/SciPy) only for the small dense factorizations the paper itself
hands to LAPACK (Sec. 2.6), and the algorithms written step by step in the
order of the paper's figures.

Modules
-------
tree      binary index tree, heap numbering (Sec. 2.7, Fig. 1)
philox    Philox4x32-10 counter-based generator and the Gaussian test matrices
          (Salmon et al., SC'11; randomized sampling of Sec. 2.5)
lowrank   qr / svd / id in the paper's three modes (Secs. 2.2-2.4, 2.6)
hodlr     HODLR compression, Fig. "Randomized compression of a HODLR matrix"
          (Sec. 3), level-truncated apply A^(l) (Sec. 2.8)
hbs       HBS compression (Figs. basic / storage-efficient HBS, Sec. 4.1-4.2),
          partial apply (Fig. "Application of A^(m) in the HBS framework"),
          HBS-ID conversion with adaptive rank (Fig. HBS-ID, Sec. 4.3)
grad      factored HODLR apply, its transpose and the gradients of
          ||Hx - b||^2 with respect to x, U, V, D
metrics   relative Frobenius error and the randomized estimate E (Sec. 5)
cost      operation counts of the oracle's own arithmetic (T_net, Sec. 5)

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test except where the docstring says
"parity unpinned".
"""
