"""FP64 CPU oracle for the fast inverse-multiquadric matrix-vector product.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call, link or execute anything in this package.  The product path (the CUDA
library and its Python binding) never touches it and shares no code with it.

Contents, each following the paper (De Marchi, Egidi, Giacomini, Maponi,
Perticarini, "Computational issues by interpolating with inverse
multiquadrics: a solution", arXiv 2205.04194):

* ``dense``      -- plain definition of b = A u, A_ij = 1/sqrt(|x_i-x_j|^2+c^2)
                    (Section 2, Eq. (4)-(5)), plus dA/dc and off-node evaluation.
                    The inner loop is plain C (OpenMP over rows), FP64.
* ``harmonics``  -- associated Legendre functions, the truncated spectral series
                    of the Laplace Green's function (Eqs. (7)-(8)), the bound of
                    Theorem 2.1 (Eq. (9)), regular/irregular solid harmonics.
* ``treecode``   -- Algorithm 1 of Section 2.2 taken step by step (uniform
                    levels from 4x4, moments v_k/w_k, far field on S_p, near
                    field on NS_p at the finest level).
* ``tree``       -- Morton quantisation, stable sort, adaptive quadtree and the
                    U/V/W/X interaction lists, written independently of the GPU
                    builder so that the two can be compared bit for bit.
* ``fmm``        -- FP64 complex fast multipole reference on that tree (P2M, M2M,
                    M2L, L2L, L2P, M2P, P2L, P2P).
* ``solve``      -- dense Cholesky, CG and additive-Schwarz PCG in FP64.
* ``grad``       -- validation-loss gradient w.r.t. c and the data values.
"""
