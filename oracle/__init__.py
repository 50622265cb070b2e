"""FP64 CPU oracle of the gDC step for rigid multiblob suspensions.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, dense restatement
of Westwood, Delmotte & Keaveny, "A generalised drift-correcting time
integration scheme for Brownian suspensions of rigid particles with
arbitrary shape" (arXiv 2106.00449), written in NumPy FP64 so that a reader
can check it against the paper by eye.  It exists to check the CUDA library
and is imported only by the tests, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg.  The library never imports, links or executes
anything from here, and this package imports nothing from the library.

Modules
-------
geometry   quaternions, rotation matrix, exp map, blob positions (Sec. 2, App. A)
rpy        dense Rotne-Prager-Yamakawa blob mobility M (Sec. 4.1)
rigid      K, K^T K, saddle-point solve, body mobility N, least squares (Sec. 2.2, 3, 5)
forces     soft blob-blob repulsion between different bodies (Eq. soft_sphere_potential form)
philox     Philox4x32-10 counter-based generator and Box-Muller normals
gdc        the gDC step (Sec. 3, RFD and FD divergence) and Euler-Maruyama (App. D)
matfree    matrix-free selected rows of M lambda for sizes too large to store M

Parity status: every function is pinned by a CPU test against closed forms,
invariants, library special cases or brute force, except the per-sample
gDC trajectory itself, for which the paper prints no worked example; it is
pinned through its exact covariance identity and its first and second
moments (App. E) instead.
"""
