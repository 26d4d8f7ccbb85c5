"""FP64 CPU oracle for the Faceted HyperSARA PDFB iteration (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite, the smoke check of ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it.  It is a plain, slow, step-by-step restatement of
the method in float64/complex128 with numpy and scipy primitives (FFT, sparse
matrix-vector products, dense SVD/eigh), written from the paper:

* ``nufft``    measurement operator Phi_l = Theta_l G_l F Z (Sec. 2.1, Eq. 1),
               w-projection rows of G (Sec. 3.2), brute-force NUDFT, power
               iteration and ARPACK Lanczos for ||Phi_l||^2.
* ``wavelets`` Daubechies filters by spectral factorisation, the SARA
               dictionary (Dirac + db1..db8) and its exact faceted form
               (Sec. 2.2.2, spatial faceting).
* ``prox``     l2-ball projection (Eq. 2), weighted l21 prox, weighted
               singular-value soft-thresholding, nuclear facets.
* ``pdfb``     the primal-dual forward-backward iteration for Eq. 3 with
               reweighting (Sec. 2.2.3).
* ``defaults`` PSF-peak normalisation, residual and dirty image (Sec. 5.3),
               dirty-image defaults of mu and mu_bar (a reading: the paper
               defers the heuristics to Part I).
* ``reduction`` visibility-gridding data reduction: gridding operator
               Gamma = Lambda G^H Theta^H, reduced operator Phi' = Lambda H F Z
               (Sec. 3.4, Eqs. 4-5), the default bound eps' (a reading).
* ``adaptive`` adaptive estimation of the effective noise level during the
               first PDFB iterations (Sec. 3.3 (ii); the schedule is a
               reading built from the Sec. 3.3 (i) estimator and Eq. 2).

Nothing here is shared with the CUDA library; the two implementations are
compared in the tests.  Every function states the passage it follows and,
where the paper is silent, the reading it takes.

Parity status: the iterate after k PDFB steps (``pdfb.run``) is "parity
unpinned" against the paper itself, which prints no iterate; it is pinned by
fixed-point, feasibility and special-case properties only.
"""
