"""Oracle: a plain, slow, FP64 CPU implementation of the paper's method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import,
call, link or execute anything under ``oracle/``.  The CUDA product path in
``paper_2603_19647_gb300`` never imports it and shares no code with it: the
two meet only through the seeded input generators, which hold none of the
method's arithmetic.

Modules (each function cites the passage of Liu & Peng, "On-the-fly ROM-based
acceleration of SI-DSA for implicit time marching of the RTE", it follows):

* ``quadrature``  Gauss-Legendre slab rule and Chebyshev-Legendre rule (Sec. 2.1, App. A).
* ``transport``   Q0 and Q1 upwind DG sweeps + moment (Sec. 2.1 Eq. (DG), Sec. 2.2, Sec. 2.3), via plain C loop nests.
* ``dsa``         diffusion correction operators (Q0 cell-centred; Q1 interior penalty) and conjugate
                  gradients (Sec. 2.3 Eq. (rho_residual)).
* ``sisa``        memory-efficient SI-SA, Algorithm 1.
* ``rom``         incremental SVD (App. B) and the DMD reduced operators (Sec. 3.1, 3.2).
* ``stepper``     the on-the-fly ROM-accelerated time march, Algorithm 2.
* ``dense``       a direct solve of the implicit system Eq. (kinetic_dg_discrete) on tiny grids.

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except where its docstring says "parity unpinned".
"""
