"""Plain, slow CPU FP64 oracle for two-site ab initio DMRG (arXiv:2311.02854).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The CUDA library never calls it and shares no code with it; the only
common module is ``synthetic_inputs`` (seeded input generators).

Modules
-------
hamiltonian  spin-orbital integrals, Fock-space operators, determinant FCI
             (the exact references every other part is pinned to)
blocks       block-sparse operators, the local basis, the normal and
             complementary operators of Sec. 2.3, blocking of a block with a
             site, and the renormalisation of Eq. (Renorm)
sigma        the two-site sigma vector of Eq. (Sigma) and the diagonal of H_eff
dmrg         environments, Davidson, decimation and the two-dot sweep

Conventions (the paper leaves them implicit):
spin orbital p = 2*i + s (s = 0 alpha, 1 beta), Jordan-Wigner order
(1a, 1b, 2a, 2b, ...); local basis {vac, b, a, ab} with |ab> = a+_a a+_b |vac>;
<pq|rs> = (i_p i_r | i_q i_s) delta(s_p, s_r) delta(s_q, s_s) and
w_pqrs = <pq||rs> = <pq|rs> - <pq|sr>; the Hamiltonian is Eq. (Hsq).

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
closed forms, brute-force Fock-space algebra or FCI; none is "parity unpinned"
except where its docstring says so.
"""
