"""FP64 CPU oracle for the extended-stencil FDTD method (Blinne et al., 1710.06829).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
calls it, and the oracle shares no code with that path.

Modules
-------
``dispersion``  numerical dispersion relation (Sec. 3, App. B), the dispersion
                norm (Sec. 4, Eq. norm) with its closed-form gradient, the exact
                CFL time-step limit (Eq. constraints) and the SLSQP coefficient
                minimiser (Sec. 4).
``fdtd``        leapfrog stepping on the staggered grid (Sec. 2, App. A update
                equations), its hand-written adjoint with the coefficient
                gradient, the divergence diagnostics (Sec. 2.1/2.2) and the
                rigid-bunch current that satisfies the discrete continuity
                equation (App. A).
``pic``         macro-particles coupled to the solver: first-order shape, staggered
                field gather, Boris push and Esirkepov's charge-conserving current
                (App. A, numerical continuity equation), one leapfrog PIC cycle.

Units throughout: c = 1, mu0 = eps0 = 1.
"""
