"""CPU oracle for the FETI interface solve of the coupled poroelasticity/elasticity model.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import anything from
this package.  The CUDA library never calls it, links it or shares code with it.

The oracle is a plain, slow, FP64 restatement of Ge & Wang, "A Parallel Solver with
Multiphysics Finite Element Method for Poroelasticity Coupled with Elasticity Model"
(arXiv 2509.06673):

* ``quadrature``  -- triangle quadrature rules (load rule of degree 5, exact rules).
* ``mesh``        -- structured right-triangle meshes per subdomain, node keys (Sec. 2.4).
* ``fem``         -- P1/P2 element matrices of the bilinear forms of Eq. (2.21)-(2.23).
* ``problem``     -- parameters, the closed-form solution of Test Case 1 (Sec. 4.1) and
                     its sources, Barry-Mercer data (Sec. 4.3), point source.
* ``local``       -- the 4-field per-subdomain block of the system in Sec. 2.5
                     (u, xi, eta, p) and the 2-field elastic block (u, xi).
* ``jump``        -- the signed Boolean jump operator B (H_P, -H_E of Sec. 2.5),
                     rigid modes and the coarse matrix G.
* ``monolithic``  -- the full saddle system of Sec. 2.5 solved by sparse LU.
* ``feti``        -- the FETI solve of Sec. 3 (Algorithm 1 with the Dirichlet
                     preconditioner of Eq. (3.5)) plus the FETI-1 coarse projection,
                     and preconditioned MINRES where the interface operator is
                     indefinite (pressure multipliers between poroelastic subdomains).
* ``errors``      -- L2 errors against the closed-form solution (Tables 3 and 4).

Parity status of each function is stated in its module header; every function is pinned
by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py`` unless it says "parity unpinned".
"""
