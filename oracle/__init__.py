"""FP64 CPU oracle for the cosine-product Krylov solvers of El Ichi, El Guide and
Jbilou, "Discrete cosine transform LSQR and GMRES methods for multidimensional
ill-posed problems" (arXiv 2103.11847).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The CUDA library never calls it, and it shares no code with the CUDA path.

Everything here is plain NumPy in float64. A library primitive (a matmul, an
SVD, a linear solve) may serve as one step; there is no blocking or fusion.

Tensor layout: a third-order tensor X in R^{n1 x n2 x n3} is a NumPy array of
shape (n3, n1, n2), so ``X[k]`` is the k-th frontal slice X(:, :, k).

Modules:
  cproduct    -- §2.1-§2.2: DCT matrix, th(v), mat/ten, the c-product
                 (Definition 2.1) and the transform route (Algorithm 1 with
                 the mode-3 matrix M of Remark 2.1), its adjoint, <.,.>.
  krylov      -- §3: Algorithm 2 (Arnoldi), Algorithm 3 (DC-GMRES(m)),
                 Algorithm 4 (Golub-Kahan), Algorithm 5 (DC-GK),
                 Algorithm 6 (DC-LSQR).
  regularize  -- §3.1 eqs. (leastsq), (tikho2), (gcv2); §3.2 (normeq2):
                 the projected Tikhonov problem and the GCV choice of lambda.
  metrics     -- §4: relative error and SNR.

Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (closed forms, the explicit block Toeplitz-plus-Hankel
definition, library routines, brute force); see tests/test_oracle_*.py.
"""
