"""Plain FP64 CPU oracle for the DD-alpha-AMG multilevel solver (arXiv:1307.6101).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or calls it, and it never
imports the CUDA library.

Every function restates one step of the method in numpy, in the order and
notation of the paper (Frommer, Kahl, Krieg, Leder, Rottmann, "An adaptive
aggregation based domain decomposition multilevel method for the lattice
Wilson Dirac operator: multilevel results"):

* ``lattice``   -- geometry, shifts with boundary signs, lattice blocks;
* ``gamma``     -- Dirac matrices in a chiral basis with Gamma_5 = diag(1,1,-1,-1);
* ``wilson``    -- Wilson-clover operator D (Sec. 1, the gamma_5-symmetric D);
* ``stencil``   -- nearest-neighbour block stencils (the coarse operators D_l);
* ``transfer``  -- block-spin aggregation P_l, R = P_l^dagger, D_{l+1} = P^dagger D P (Sec. 1, 2);
* ``smoother``  -- minimal residual block solver and SAP (Sec. 1, Table 1);
* ``krylov``    -- FGMRES / GMRES and the even-odd coarsest solve (Sec. 2.1, 3);
* ``multigrid`` -- V-/K-cycle (Alg. 1, Alg. 2) and the setup (Alg. 3, Alg. 4);
* ``spectrum``  -- smallest singular value of D and the m0 bisection used to
  pick the benchmark masses.

Parity status: everything is pinned by tests under ``tests/`` against closed
forms, invariants or brute force, except where a module header says
"parity unpinned".
"""
