"""Oracle: a plain, slow, obviously correct FP64 / exact-integer CPU statement of
what the GPU path computes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path under ``paper_2510_04795_gb300/`` never imports it
and shares no code with it; both take their inputs from ``synthetic``.

Modules (each function cites the passage of the paper it follows):

* ``ozaki``    exact Ozaki-scheme emulation of C = AB (section "Theory of
               emulated FP64 arithmetic"; slice/bit relation in "Numerical
               procedure").
* ``heff``     block-sparse two-site H_eff * psi, plain FP64 per block, a dense
               Kronecker brute force, and the emulated two-stage definition.
* ``fci``      exact diagonalisation (full CI) of the ab initio Hamiltonian.
* ``davidson`` Davidson eigensolver (the Krylov step of the DMRG update).
* ``dmrg``     explicit-basis two-site DMRG sweep.

Parity status of every function is stated in its module header.
"""
