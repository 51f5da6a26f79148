"""CPU FP64 oracle for the treecode-accelerated boundary-element
Poisson-Boltzmann method of Cooper & Barba (arXiv 1506.03745).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants generator with the CUDA library; the only thing
both sides consume is the seeded input generator module ``synth``.

Modules (each function cites the passage of the paper it restates):
  units       -- CODATA constants and the internal unit system (Section 2).
  quadrature  -- symmetric triangle rules derived from their moment equations
                 and Gauss-Legendre rules (Section 3.1).
  geometry    -- flat-panel geometry: centroids, normals, areas, L (Section 3.1).
  integrals   -- Laplace/Yukawa kernels, the three-tier panel integration and
                 the semi-analytical self integral (Eq. 8-9, Section 3.1).
  bem         -- dense assembly of the block systems (Eq. 6, Eq. 7 and the
                 single-molecule 2x2 block), LU solve, direct-sum matvec.
  energy      -- Coulomb, solvation, surface, total and interaction energies
                 (Eq. 11-17).
  analytical  -- the two-sphere Legendre-series solution (Section 4) and its
                 isolated-body limits.
  treecode    -- octree, multipole-acceptance lists and the truncated Cartesian
                 Taylor expansion evaluated by univariate power series
                 (Section 3.2).
  regions     -- more interfaces (Stern layers, solvent-filled cavities: the
                 extension stated after Eq. 7) as per-region rows, their
                 treecode product, and the closed forms that pin them.

Parity status: every function is pinned by a test in tests/test_oracle_*.py
except where its docstring says "parity unpinned".
"""
