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


def _group_with_singular_values(s, forward, seed=5):
    """One quantum-number group whose matrix M_q has the singular values s
    (two column blocks forward, two row blocks backward), as a layout + vector."""
    rng = np.random.default_rng(seed)
    nr, nc = (6, 9) if forward else (9, 6)
    U, _ = np.linalg.qr(rng.standard_normal((nr, nr)))
    V, _ = np.linalg.qr(rng.standard_normal((nc, nc)))
    r = len(s)
    M = (U[:, :r] * s) @ V[:, :r].T
    if forward:
        # left sector 0 with c1 = 0 (label (0,0)); column components (c2, ir) = (0, 0), (1, 1)
        layout = [(0, 0, 0, 0, 0, 6, 5), (0, 0, 1, 1, 30, 6, 4)]
        psi = np.concatenate([M[:, :5].ravel(), M[:, 5:].ravel()])
        left, right = [(0, 0)], [(0, 0), (1, -1)]
    else:
        # right sector 0 with c2 = 0; row components (il, c1) = (0, 0), (1, 0)
        layout = [(0, 0, 0, 0, 0, 5, 6), (1, 0, 0, 0, 30, 4, 6)]
        psi = np.concatenate([M[:5].ravel(), M[5:].ravel()])
        left, right = [(0, 0), (0, 0)], [(0, 0)]
    return layout, psi, left, right, M


@pytest.mark.parametrize("forward", [True, False])
def test_decimation_near_null_singular_values_match_svd(forward):
    """One root: the weights are the squared singular values of M_q, including
    values far below the rounding floor of a density-matrix eigensolver
    (1e-10, 1e-13), and exactly singular directions are dropped (s <= 1e-14)."""
    s = np.array([1.0, 0.5, 1e-3, 1e-10, 1e-13])  # rank 5 of 6: one exact zero
    layout, psi, left, right, M = _group_with_singular_values(s, forward)
    groups, kept, w = decimate(layout, psi[None, :], left, right, 10, forward)
    assert len(kept) == 1
    q, vec, _ = kept[0]
    assert vec.shape[1] == 5  # the exactly singular direction is not kept
    ref = np.linalg.svd(M, compute_uv=False)
    assert abs(ref[5]) < 1e-14
    assert w < 1e-28
    # the kept vectors span the leading singular subspace of M_q
    Uref, sref, Vtref = np.linalg.svd(M)
    basis = Uref[:, :5] if forward else Vtref[:5].T
    np.testing.assert_allclose(np.abs(vec.T @ basis), np.eye(5), atol=1e-6)
    # truncation to D = 2: the discarded weight is the sum of the dropped s^2
    _, kept2, w2 = decimate(layout, psi[None, :], left, right, 2, forward)
    assert kept2[0][1].shape[1] == 2
    assert abs(w2 - np.sum(s[2:] ** 2)) < 1e-18
