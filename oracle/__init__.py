"""CPU oracle for the shifted-COCG / Dyson transport path (TEST INFRASTRUCTURE).

This package is a plain, slow, FP64 restatement of what the method computes,
written from the paper (Iwase, Hoshi, Ono, "Efficient numerical solver for
first-principles transport calculation based on real-space finite-difference
method") and used only to check the CUDA library.  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import or run it; the library itself never does, and shares
no code with it.  The only common module is ``workloads`` (seeded inputs, no
method arithmetic).

Modules and the passages they follow:

* ``operator``      -- the RSFD Hamiltonian H_T (Sec. II A, Eq. sabun1 and the
                       block-tridiagonal matrix that follows it) and the
                       boundary row set.
* ``cocg``          -- conventional COCG and shifted COCG with seed switching
                       (Appendix: Eqs. Eq, xvec, rvec, pvec, alpha, beta,
                       collinear, spi, salpha, sbeta, endcollinear,
                       seedswitch).
* ``dense``         -- dense resolvents (Eqs. GF1, GF2, GF4) on tiny grids.
* ``leads``         -- lead self-energies (Eqs. self-energy,
                       surface green's function, sec2-01, sec2-02) for a
                       uniform V=0 finite-difference lead, by Bloch roots
                       and by Sancho-Rubio decimation, and for a lead that
                       repeats one principal layer with its own potential
                       (decimation).
* ``dyson``         -- unperturbed -> perturbed boundary Green's function
                       (Eq. sec3-01a as a linear solve, and the block
                       formulas Eqs. sec3-02 ... sec3-06).
* ``transmission``  -- Fisher-Lee transmission (Eq. TF and the definition
                       of Gamma that follows it).

Pins: every function is checked in ``tests/test_oracle_*.py`` against
something other than itself (dense inversion by a library routine, closed
forms, polynomial exactness of the finite-difference stencil, integer channel
counts, symmetry).  No function here is parity-unpinned.
"""
