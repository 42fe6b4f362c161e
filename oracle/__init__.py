"""CPU oracle of the quadrature-free ADER-AFE-DG step (FP64, plain loops over cells).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (the C-ABI library and its Python binding) never calls it and
shares no code with it: this package has its own reference-element algebra
(exact rationals), its own mesh topology and its own scheme, written from the
paper's Sec. 4 and App. A.

Modules
-------
``refelem``  reference P_N basis, universal matrices, time basis (Sec. 4.1, 4.3, App. A)
``mesh``     per-cell AFE nodes, Jacobians, mass matrices, faces (Sec. 4.1, 4.3, 4.4)
``scheme``   time step, limiter, predictor, Rusanov fluxes, corrector (Sec. 4.2-4.5)
``density_wave_run``  command-line full-length run of the density-wave accuracy case

Parity pinning: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute-force quadrature, invariants or values printed in
the paper; none is "parity unpinned".
"""
