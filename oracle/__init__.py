"""CPU oracle for EA/IP-ADC(n) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU path.

Tiers:
  fock.py        T0: operator definitions evaluated by brute force in Fock space.
  spinorb.py     T1: explicit spin-orbital working equations (dense integrals).
  spinadapted.py T2: spin-adapted, density-fitted working equations (matrix-free).
  davidson.py    dense / Davidson eigensolvers, spin-adapted metric, spectroscopic factors.
"""
