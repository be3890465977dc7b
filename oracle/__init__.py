"""FP64 CPU oracle for the MAC Navier-Stokes / Newton / FGMRES / PLMM-preconditioner path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement of the
method (arXiv 2510.22077) in NumPy + SciPy sparse, double precision throughout.  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  The GPU library never links, imports or calls it, and it imports
nothing from the GPU package.

Modules
    mac     -- grid, unknowns, pressure pins, residual r(x) and Jacobians as CSR  (Eq. 1-3, Sec. 2, Eq. 27)
    maps    -- primary grids, contact interfaces, face classes, dual grids, gPLMM tags  (Sec. 3.2.1, 4)
    plmm    -- preconditioner build and apply, recipe form and literal matrix form  (Eqs. 5-26)
    krylov  -- right-preconditioned flexible GMRES, Newton, backward-Euler stepping  (Sec. 8, Eq. 3)
    block   -- block-triangular Schur comparator with the scaled BFBt approximation  (Sec. 1, Eq. 4)
    unet    -- 3D U-Net of the learned initial guess: NumPy forward and explicit backward, sample encoding
    coarse_solver -- coarse-scale Navier-Stokes solver: Newton on the coarse unknowns  (Sec. 5, Alg. 1)

Parity status: every function is pinned by a test in tests/test_oracle_*.py against something
other than itself (closed forms, finite differences, brute-force dense solves, the projection
property of M_G, single-subdomain exactness, two independent formulations of M_G and M).  The
FGMRES/Newton iteration COUNTS have no pin (the paper prints them only in figures): parity unpinned.
"""
