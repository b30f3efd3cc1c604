"""FP64 CPU oracle for the ADER-DG + clustered-LTS update (test infrastructure).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (the C-ABI library and its Python binding) never imports,
links or calls anything here, and this package imports nothing from the product.

It is a plain, slow, obviously-correct restatement of the method of
"Next-Generation Local Time Stepping for the ADER-DG Finite Element Method"
(Breuer & Heinecke), following the paper's own order and notation:

* ``basis``   -- modal orthonormal tetrahedral basis (Sec. III-A, Karniadakis-Sherwin
                 expansion), Gauss quadrature, reference operators K_c, F~_i, F^_i,
                 F-_{j,h} (Sec. III-A "Volume/Surface Kernel").
* ``mesh``    -- element geometry, face neighbours and the (j, h) relation (Sec. III-A).
* ``physics`` -- Jacobians of Eq. (1), anelastic coupling E / E', relaxation fit,
                 star matrices and upwind flux solvers (Sec. III-A).
* ``lts``     -- CFL time steps, rate-2 clustering, normalisation and the lambda
                 search (Sec. V-A).
* ``scheme``  -- time kernel (Eqs. ader_taylor, ader_derivative_*), volume kernel,
                 local/neighbour surface kernels, update (Eq. update), the LTS
                 buffers B1/B2/B3 and their use (Sec. V-B), global time stepping,
                 point source, receivers and the discrete energy.
* ``partitioned`` -- a run split into parts that exchange the face-local messages
                 H = X F-_{j,h} (Sec. V-C); pinned against the unpartitioned oracle.
* ``adjoint`` -- discrete adjoint of the global-time-stepping and clustered-LTS loops for
                 the seismogram misfit (Sec. VII-B) and the material derivatives of the
                 star matrices and flux solvers; pinned by central differences of the
                 oracle's own misfit.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test except where the docstring says
"parity unpinned".
"""
