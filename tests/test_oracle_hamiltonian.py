"""Pins for the integrals, the Fock-space algebra and determinant FCI."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle.hamiltonian import (SITE_CREATORS, eri_from_cholesky, fci_energies, fock_creators,
                                fock_hamiltonian, fock_number_ops, spin_orbital_integrals)


def test_integral_symmetries_and_psd():
    h, L = si.make_integrals(6, 24, seed=0)
    eri = eri_from_cholesky(L)
    assert np.allclose(h, h.T)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.allclose(eri, eri.transpose(perm))
    sup = eri.reshape(36, 36)
    assert np.linalg.eigvalsh(sup).min() > -1e-12
    assert np.allclose(np.diag(h), np.linspace(-4, 0, 6))


def test_spin_orbital_antisymmetry():
    h, L = si.make_integrals(3, 8, seed=0)
    hso, w = spin_orbital_integrals(h, eri_from_cholesky(L))
    assert np.allclose(w, -w.transpose(1, 0, 2, 3))
    assert np.allclose(w, -w.transpose(0, 1, 3, 2))
    assert np.allclose(w, w.transpose(2, 3, 0, 1))
    # spin conservation: <pq||rs> = 0 unless s_p + s_q = s_r + s_s
    n = hso.shape[0]
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    if (p % 2) + (q % 2) != (r % 2) + (s % 2):
                        assert w[p, q, r, s] == 0.0


def test_site_creators_car():
    a, b = SITE_CREATORS
    for X in (a, b):
        assert np.allclose(X @ X, 0)
        assert np.allclose(X @ X.T + X.T @ X, np.eye(4))
    assert np.allclose(a @ b + b @ a, 0)
    assert np.allclose(a @ b.T + b.T @ a, 0)
    # |ab> = a+_a a+_b |vac>
    vac = np.eye(4)[:, 0]
    assert np.allclose(a @ b @ vac, np.eye(4)[:, 3])


def test_fock_car_and_number():
    K = 3
    cd = fock_creators(K)
    n = len(cd)
    for p in range(n):
        for q in range(n):
            ac = (cd[p].T @ cd[q] + cd[q] @ cd[p].T).toarray()
            assert np.allclose(ac, np.eye(4 ** K) * (p == q))
            cc = (cd[p] @ cd[q] + cd[q] @ cd[p]).toarray()
            assert np.allclose(cc, 0)
    N, S = fock_number_ops(K, cd)
    assert N.diagonal().max() == 2 * K


def test_fci_closed_form_no_interaction():
    h, L = si.make_integrals(6, 8, seed=3)
    eri = 0.0 * eri_from_cholesky(L)
    ev = np.linalg.eigvalsh(h)
    for N, twoS in [(6, 0), (5, 1), (4, 2)]:
        na, nb = (N + twoS) // 2, (N - twoS) // 2
        e = fci_energies(h, eri, N, twoS)[0]
        assert abs(e - (ev[:na].sum() + ev[:nb].sum())) < 1e-12


def test_fci_matches_fock_space():
    """Determinant FCI and the Fock-space H (independent constructions)."""
    K, N, twoS = 4, 4, 0
    h, L = si.make_integrals(K, 16, seed=0)
    eri = eri_from_cholesky(L)
    hso, w = spin_orbital_integrals(h, eri)
    cd = fock_creators(K)
    H = fock_hamiltonian(hso, w, cd)
    assert abs(H - H.T).max() < 1e-12
    Nop, Sop = fock_number_ops(K, cd)
    idx = np.where((np.abs(Nop.diagonal() - N) < 1e-9) & (np.abs(Sop.diagonal() - twoS) < 1e-9))[0]
    e_fock = np.linalg.eigvalsh(H[idx][:, idx].toarray())[:4]
    e_fci = fci_energies(h, eri, N, twoS, 4)
    assert np.allclose(e_fock, e_fci, atol=1e-11)


def test_fci_size_consistency():
    """Two decoupled subsystems: E = E_A + E_B (block-diagonal h and L)."""
    hA, LA = si.make_integrals(3, 6, seed=4)
    hB, LB = si.make_integrals(3, 6, seed=5)
    h = np.zeros((6, 6))
    h[:3, :3], h[3:, 3:] = hA, hB
    L = np.zeros((12, 6, 6))
    L[:6, :3, :3], L[6:, 3:, 3:] = LA, LB
    eA = fci_energies(hA, eri_from_cholesky(LA), 2, 0)[0]
    eB = fci_energies(hB, eri_from_cholesky(LB), 2, 0)[0]
    e = fci_energies(h, eri_from_cholesky(L), 4, 0)
    # the ground state of the union with 4 electrons: the best split of electrons
    best = min(
        fci_energies(hA, eri_from_cholesky(LA), nA, sA)[0] + fci_energies(hB, eri_from_cholesky(LB), 4 - nA, -sA)[0]
        for nA in range(0, 5) for sA in range(-nA, nA + 1, 2)
        if abs(sA) <= min(nA, 6 - nA) and abs(sA) <= min(4 - nA, 6 - 4 + nA) and 4 - nA <= 6
    )
    assert abs(e[0] - best) < 1e-10
    assert best <= eA + eB + 1e-12


def test_fci_sz_multiplet():
    """Levels of the 2Sz=2 sector appear in the 2Sz=0 spectrum (S^- symmetry)."""
    h, L = si.make_integrals(4, 12, seed=0)
    eri = eri_from_cholesky(L)
    e2 = fci_energies(h, eri, 4, 2, 3)
    e0 = fci_energies(h, eri, 4, 0, 36)
    for e in e2:
        assert np.min(np.abs(e0 - e)) < 1e-10


def test_golden_fci_values_reproduce():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.txt")
    for line in open(path):
        if line.startswith("#"):
            continue
        head, vals = line.split(":")
        name, K, N, twoS, nc, ell, hmin = head.split()
        if int(K) > 6:
            continue
        h, L = si.make_integrals(int(K), int(nc), ell=float(ell), h_min=float(hmin), seed=0)
        e = fci_energies(h, eri_from_cholesky(L), int(N), int(twoS), len(vals.split()))
        assert np.allclose(e, [float(v) for v in vals.split()], atol=1e-11)
