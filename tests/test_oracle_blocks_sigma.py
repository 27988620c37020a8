"""Pins for the block algebra, renormalisation, sigma and diag(H_eff).

Every renormalised operator and every sigma vector is compared with its Fock-space
definition B^T O B, where B holds the block basis vectors built directly from
the MPS tensors (``left_block_vectors`` / ``right_block_vectors``)."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import blocks as ob
from oracle.dmrg import Oracle
from oracle.hamiltonian import (eri_from_cholesky, fock_creators, fock_hamiltonian,
                                left_block_vectors, right_block_vectors, spin_orbital_integrals)


def _problem(K=5, N=5, twoS=1, D=10, center=3, seed=2):
    h, L = si.make_integrals(K, 4 * K, seed=0)
    eri = eri_from_cholesky(L)
    bonds = si.bond_sectors(K, N, twoS, D)
    mps = si.random_mps(K, N, twoS, bonds, center=center, seed=seed)
    return h, eri, mps


def _fock_ops(h, eri, nsites, offset):
    """Fock-space operators of a block of ``nsites`` sites whose first spin
    orbital is ``offset`` (JW strings inside the block only)."""
    hso, w = spin_orbital_integrals(h, eri)
    cd = fock_creators(nsites)
    return hso, w, {offset + i: c for i, c in enumerate(cd)}


def _embed(V, basis):
    """Dense basis matrix of a block from {sector: vectors} in basis order."""
    return np.hstack([V[i] for i in range(len(basis.qn))])


def _check_block(X, V, cd, hso, w, tol=1e-12):
    Bm = _embed(V, X.basis)
    an = {p: c.T for p, c in cd.items()}

    def proj(op):
        return Bm.T @ (op @ Bm)

    for p in X.orbs:
        assert np.abs(X.C[p].dense() - proj(cd[p].toarray())).max() < tol
    for (p, q), A in X.A.items():
        assert np.abs(A.dense() - proj((cd[p] @ cd[q]).toarray())).max() < tol
    for (p, s), B in X.B.items():
        assert np.abs(B.dense() - proj((cd[p] @ an[s]).toarray())).max() < tol
    orbs = X.orbs
    for p in X.others:
        S = 0
        for q in orbs:
            S = S + 0.5 * hso[p, q] * an[q]
            for i, s in enumerate(orbs):
                for r in orbs[i + 1:]:
                    S = S + w[p, q, s, r] * (cd[q] @ an[r] @ an[s])
        ref = proj(S.toarray()) if not np.isscalar(S) else 0
        assert np.abs(X.S[p].dense() - ref).max() < tol, p
    Hf = 0
    for p in orbs:
        for q in orbs:
            Hf = Hf + hso[p, q] * (cd[p] @ an[q])
    for i, p in enumerate(orbs):
        for q in orbs[i + 1:]:
            for j, s in enumerate(orbs):
                for r in orbs[j + 1:]:
                    Hf = Hf + w[p, q, s, r] * (cd[p] @ cd[q] @ an[r] @ an[s])
    assert np.abs(X.H.dense() - proj(Hf.toarray())).max() < tol
    # complementary operators formed from A and B
    for p in X.others[:3]:
        for q in X.others[-3:]:
            P = 0
            for i, s in enumerate(orbs):
                for r in orbs[i + 1:]:
                    P = P + w[p, q, s, r] * (an[r] @ an[s])
            Q = 0
            for qq in orbs:
                for r in orbs:
                    Q = Q + w[p, qq, q, r] * (cd[qq] @ an[r])
            assert np.abs(X.P(p, q).dense() - proj(P.toarray())).max() < tol
            assert np.abs(X.Q(p, q).dense() - proj(Q.toarray())).max() < tol


@pytest.mark.parametrize("m", [1, 2, 3])
def test_left_block_operators_are_projections(m):
    h, eri, mps = _problem(center=4)
    o = Oracle(h, eri, mps.N, mps.twoS, mps)
    X = o.left_block(m)
    hso, w, cd = _fock_ops(h, eri, m, 0)
    _check_block(X, left_block_vectors(mps, m), cd, hso, w)


@pytest.mark.parametrize("m", [4, 3, 2])
def test_right_block_operators_are_projections(m):
    h, eri, mps = _problem(center=1)
    o = Oracle(h, eri, mps.N, mps.twoS, mps)
    Y = o.right_block(m)
    hso, w, cd = _fock_ops(h, eri, mps.K - m, 2 * m)
    _check_block(Y, right_block_vectors(mps, m), cd, hso, w)


def _superblock_basis(mps, k, ts):
    VL = left_block_vectors(mps, k - 1)
    VR = right_block_vectors(mps, k + 1)
    Bm = np.zeros((4 ** mps.K, ts.dim))
    for (il, c1, c2, ir, off, dl, dr) in ts.layout:
        mid = np.kron(np.eye(4)[c1], np.eye(4)[c2])
        for a in range(dl):
            left = np.kron(VL[il][:, a], mid)
            for b in range(dr):
                Bm[:, off + a * dr + b] = np.kron(left, VR[ir][:, b])
    return Bm


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_sigma_equals_projected_fock_hamiltonian(k):
    h, eri, mps = _problem(center=k)
    o = Oracle(h, eri, mps.N, mps.twoS, mps)
    ts = o.two_site(k)
    hso, w = spin_orbital_integrals(h, eri)
    H = fock_hamiltonian(hso, w)
    Bm = _superblock_basis(mps, k, ts)
    assert np.abs(Bm.T @ Bm - np.eye(ts.dim)).max() < 1e-12
    Heff = Bm.T @ (H @ Bm)
    for seed in (1, 7):
        psi = si.random_vector(ts.dim, seed=seed)
        s = ts.sigma(psi)
        ref = Heff @ psi
        assert np.linalg.norm(s - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.abs(ts.hdiag() - np.diag(Heff)).max() < 1e-12


def test_sigma_hermitian():
    h, eri, mps = _problem(K=6, N=6, twoS=0, D=20, center=3)
    o = Oracle(h, eri, mps.N, mps.twoS, mps)
    ts = o.two_site(3)
    a = si.random_vector(ts.dim, seed=1)
    b = si.random_vector(ts.dim, seed=2)
    assert abs(a @ ts.sigma(b) - b @ ts.sigma(a)) < 1e-12


def test_planted_sign_error_is_caught(monkeypatch):
    """Dropping the fermionic factor zeta from the product rule breaks the
    Fock-space pin (the pins are sensitive to a sign slip)."""
    h, eri, mps = _problem(center=2)
    hso, w = spin_orbital_integrals(h, eri)
    H = fock_hamiltonian(hso, w)
    orig = ob.kron

    def no_zeta(PB, OX, OY):
        out = orig(PB, OX, None if OY is None else OY)
        return out if OY is None or OY.parity == 0 else _flip_odd_sectors(PB, out)

    def _flip_odd_sectors(PB, op):
        # undo the (-1)^{n(x)} factor for odd O^Y: recompute without it
        res = ob.Op(PB, op.dq, {})
        for i, blk in op.blocks.items():
            blk = blk.copy()
            for (ix, iy), off in PB.comp_off[i].items():
                if PB.BX.n(ix) & 1:
                    d = PB.BX.dim[ix] * PB.BY.dim[iy]
                    blk[:, off:off + d] *= -1.0
            res.blocks[i] = blk
        return res

    monkeypatch.setattr(ob, "kron", no_zeta)
    o = Oracle(h, eri, mps.N, mps.twoS, mps)
    ts = o.two_site(2)
    Bm = _superblock_basis(mps, 2, ts)
    psi = si.random_vector(ts.dim, seed=1)
    ref = Bm.T @ (H @ (Bm @ psi))
    assert np.linalg.norm(ts.sigma(psi) - ref) > 1e-3 * np.linalg.norm(ref)
