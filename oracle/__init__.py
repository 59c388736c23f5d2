"""FP64 CPU oracle of Sparse Frequent Directions (Ghashami, Liberty, Phillips).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product (the CUDA library and its Python binding) never imports
it, and this package imports nothing from the product.

Modules
-------
philox   Philox4x64-10 counter-based generator and the Gaussian draws the
         method makes (G in Alg. 1, x in Alg. 6).
sfd      The method itself: Alg. 1-6 plus the classical FrequentDirections
         baseline of Sec. 3.1.
metrics  Error measures of Sec. 5 (cov-err, proj-err) and the bounds of
         Sec. 2 / Lemma 3.1 / Theorem 4.1.

Every function is plain numpy / scipy in float64; library routines (matmul,
sparse matmul, QR, SVD, symmetric eigensolve) serve as single steps.
"""
