"""Pins for Davidson, decimation and the sweep: full-D DMRG equals FCI."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle.dmrg import Oracle, davidson, decimate
from oracle.hamiltonian import eri_from_cholesky, fci_energies
from oracle.sigma import two_site_layout


def test_davidson_random_symmetric():
    rng = np.random.default_rng(0)
    n = 300
    A = rng.standard_normal((n, n))
    A = A + A.T + np.diag(np.arange(n) * 0.5)
    ev = np.linalg.eigvalsh(A)
    x0 = rng.standard_normal((2, n))
    theta, X, it = davidson(lambda v: A @ v, np.diag(A).copy(), x0, n_roots=2, tol=1e-9, max_iter=500)
    assert np.allclose(theta, ev[:2], atol=1e-10)
    for i in range(2):
        assert np.linalg.norm(A @ X[i] - theta[i] * X[i]) < 1e-8


def test_decimation_keeps_largest_weights():
    rng = np.random.default_rng(1)
    left = [(0, 0), (1, 1), (1, -1)]
    right = [(2, 0), (3, 1), (3, -1), (4, 0)]
    layout, dim = two_site_layout(left, [3, 2, 2], right, [2, 3, 3, 1])
    X = rng.standard_normal((1, dim))
    X /= np.linalg.norm(X)
    groups, kept, w = decimate(layout, X, left, right, D=5, forward=True)
    sv = []
    for q, g in groups.items():
        sv += list(np.linalg.svd(g["mats"][0], compute_uv=False) ** 2)
    sv = np.sort(sv)[::-1]
    assert sum(U.shape[1] for _, U, _ in kept) == 5
    assert abs(w - sv[5:].sum()) < 1e-12
    for _, U, _ in kept:
        assert np.allclose(U.T @ U, np.eye(U.shape[1]))


def test_full_D_sweep_reproduces_fci():
    K, N, twoS = 6, 6, 0
    h, L = si.make_integrals(K, 24, seed=0)
    eri = eri_from_cholesky(L)
    efci = fci_energies(h, eri, N, twoS)[0]
    bonds = si.bond_sectors(K, N, twoS, 64)
    mps = si.random_mps(K, N, twoS, bonds, center=1, seed=2)
    E, w, be = Oracle(h, eri, N, twoS, mps).sweep(2, 64, tol=1e-8)
    assert abs(E[-1] - efci) < 1e-10
    assert np.all(w < 1e-20)


def test_truncated_sweep_is_variational():
    K, N, twoS = 6, 6, 0
    h, L = si.make_integrals(K, 24, seed=0)
    eri = eri_from_cholesky(L)
    efci = fci_energies(h, eri, N, twoS)[0]
    bonds = si.bond_sectors(K, N, twoS, 6)
    mps = si.random_mps(K, N, twoS, bonds, center=1, seed=2)
    E, w, be = Oracle(h, eri, N, twoS, mps).sweep(3, 6)
    assert np.all(be >= efci - 1e-10)
    assert w[-1] > 0
    assert E[-1] - efci < 0.05


def test_state_averaged_two_roots_full_D():
    K, N, twoS = 5, 4, 0
    h, L = si.make_integrals(K, 20, seed=0)
    eri = eri_from_cholesky(L)
    efci = fci_energies(h, eri, N, twoS, 2)
    bonds = si.bond_sectors(K, N, twoS, 64)
    mps = si.random_mps(K, N, twoS, bonds, center=1, seed=2)
    o = Oracle(h, eri, N, twoS, mps)
    E, w, be = o.sweep(2, 64, n_roots=2, tol=1e-8)
    ts, theta, X, _ = o.optimise_bond(1, si.random_vector(o.two_site(1).dim, seed=1, nvec=2), 2, 1e-9)
    assert np.allclose(theta, efci, atol=1e-9)


@pytest.mark.slow
def test_full_D_sweep_k8():
    """K=8, N=8: full D=256 reproduces the FCI energy (4900 determinants)."""
    K, N, twoS = 8, 8, 0
    h, L = si.make_integrals(K, 32, seed=0)
    eri = eri_from_cholesky(L)
    efci = fci_energies(h, eri, N, twoS)[0]
    bonds = si.bond_sectors(K, N, twoS, 256)
    mps = si.random_mps(K, N, twoS, bonds, center=1, seed=2)
    E, w, be = Oracle(h, eri, N, twoS, mps).sweep(2, 256, tol=1e-8)
    assert abs(E[-1] - efci) < 1e-10
