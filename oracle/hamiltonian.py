"""Integrals, Fock-space operators and determinant FCI (test infrastructure).

Everything here follows the plain definitions of Sec. 2.1: the Hamiltonian
Eq. (Hsq), the local basis listed after Eq. (MPS), and the Jordan-Wigner
ordering of creators.  It is the ground truth the block algebra is pinned to.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

# local basis index n = 2*n_alpha + n_beta: 0 vac, 1 beta, 2 alpha, 3 alpha-beta
_CD_ALPHA = np.zeros((4, 4))
_CD_ALPHA[2, 0] = 1.0      # a+_a |vac>  = |a>
_CD_ALPHA[3, 1] = 1.0      # a+_a |b>    = a+_a a+_b |vac> = |ab>
_CD_BETA = np.zeros((4, 4))
_CD_BETA[1, 0] = 1.0       # a+_b |vac>  = |b>
_CD_BETA[3, 2] = -1.0      # a+_b |a>    = a+_b a+_a |vac> = -|ab>
SITE_CREATORS = (_CD_ALPHA, _CD_BETA)
SITE_PARITY = np.diag([1.0, -1.0, -1.0, 1.0])


def eri_from_cholesky(L: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_X L[X,p,q] L[X,r,s]."""
    return np.einsum("xpq,xrs->pqrs", L, L, optimize=True)


def spin_orbital_integrals(h: np.ndarray, eri: np.ndarray):
    """Return (h_so, w) with w[p,q,r,s] = <pq||rs> for spin orbitals p = 2i+s."""
    K = h.shape[0]
    n = 2 * K
    hso = np.zeros((n, n))
    for s in (0, 1):
        hso[s::2, s::2] = h
    v = np.zeros((n, n, n, n))
    g = eri.transpose(0, 2, 1, 3)  # g[p,q,r,s] = (pr|qs)
    for s1 in (0, 1):
        for s2 in (0, 1):
            v[s1::2, s2::2, s1::2, s2::2] = g
    w = v - v.transpose(0, 1, 3, 2)
    return hso, w


# ---------------------------------------------------------------------------
# Fock space of K sites (tensor-product basis, site 1 most significant)
# ---------------------------------------------------------------------------

def fock_creators(K: int):
    """Sparse a+_p (p = 0..2K-1) on the 4^K Fock space with JW strings."""
    eye = sp.identity(4, format="csr")
    Z = sp.csr_matrix(SITE_PARITY)
    ops = []
    for k in range(K):
        for s in (0, 1):
            m = sp.identity(1, format="csr")
            for j in range(K):
                f = Z if j < k else (sp.csr_matrix(SITE_CREATORS[s]) if j == k else eye)
                m = sp.kron(m, f, format="csr")
            ops.append(m)
    return ops


def fock_hamiltonian(hso: np.ndarray, w: np.ndarray, cd=None):
    """H = sum h_pq a+p a_q + sum_{p<q, s<r} <pq||sr> a+p a+q a_r a_s (sparse)."""
    n = hso.shape[0]
    if cd is None:
        cd = fock_creators(n // 2)
    an = [c.T.tocsr() for c in cd]
    dim = cd[0].shape[0]
    H = sp.csr_matrix((dim, dim))
    for p in range(n):
        for q in range(n):
            if hso[p, q] != 0.0:
                H = H + hso[p, q] * (cd[p] @ an[q])
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    ann_pair = {(s, r): an[r] @ an[s] for (s, r) in pairs}   # a_r a_s
    for (p, q) in pairs:
        X = sp.csr_matrix((dim, dim))
        for (s, r) in pairs:
            c = w[p, q, s, r]
            if c != 0.0:
                X = X + c * ann_pair[(s, r)]
        if X.nnz:
            H = H + (cd[p] @ cd[q]) @ X
    return H.tocsr()


def fock_number_ops(K: int, cd=None):
    """(N, 2Sz) as sparse diagonal operators on the Fock space."""
    if cd is None:
        cd = fock_creators(K)
    dim = cd[0].shape[0]
    N = sp.csr_matrix((dim, dim))
    S = sp.csr_matrix((dim, dim))
    for p, c in enumerate(cd):
        nop = c @ c.T
        N = N + nop
        S = S + (1.0 if p % 2 == 0 else -1.0) * nop
    return N, S


# ---------------------------------------------------------------------------
# Determinant FCI in one (N, 2Sz) sector
# ---------------------------------------------------------------------------

def _strings(K: int, ne: int):
    return [sum(1 << i for i in c) for c in itertools.combinations(range(K), ne)]


def _excitation_matrices(K: int, strings):
    """E[p][q] = a+_p a_q on one spin's occupation strings (sparse)."""
    index = {s: i for i, s in enumerate(strings)}
    n = len(strings)
    E = [[None] * K for _ in range(K)]
    for p in range(K):
        for q in range(K):
            rows, cols, vals = [], [], []
            for j, s in enumerate(strings):
                if not (s >> q) & 1:
                    continue
                s1 = s & ~(1 << q)
                sign = (-1) ** bin(s & ((1 << q) - 1)).count("1")
                if (s1 >> p) & 1:
                    continue
                sign *= (-1) ** bin(s1 & ((1 << p) - 1)).count("1")
                rows.append(index[s1 | (1 << p)])
                cols.append(j)
                vals.append(float(sign))
            E[p][q] = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return E


def fci_hamiltonian(h: np.ndarray, eri: np.ndarray, N: int, twoS: int):
    """Sparse H in the determinant basis |alpha string>|beta string>.

    Spin-free form of Eq. (Hsq): H = sum h_ij E_ij + 1/2 sum (ij|kl)
    (E_ij E_kl - delta_jk E_il), with E_ij = sum_s a+_is a_js.
    """
    K = h.shape[0]
    na, nb = (N + twoS) // 2, (N - twoS) // 2
    sa, sb = _strings(K, na), _strings(K, nb)
    Ea, Eb = _excitation_matrices(K, sa), _excitation_matrices(K, sb)
    Ia, Ib = sp.identity(len(sa), format="csr"), sp.identity(len(sb), format="csr")
    E = [[sp.kron(Ea[i][j], Ib, format="csr") + sp.kron(Ia, Eb[i][j], format="csr")
          for j in range(K)] for i in range(K)]
    dim = len(sa) * len(sb)
    H = sp.csr_matrix((dim, dim))
    for i in range(K):
        for j in range(K):
            coef = h[i, j] - 0.5 * sum(eri[i, k, k, j] for k in range(K))
            G = coef * E[i][j]
            for k in range(K):
                for l in range(K):
                    if eri[i, j, k, l] != 0.0:
                        G = G + 0.5 * eri[i, j, k, l] * (E[i][j] @ E[k][l])
            H = H + G
    return H.tocsr()


def fci_energies(h: np.ndarray, eri: np.ndarray, N: int, twoS: int, nroots: int = 1):
    H = fci_hamiltonian(h, eri, N, twoS)
    if H.shape[0] <= 6000:
        return np.linalg.eigvalsh(H.toarray())[:nroots]
    import scipy.sparse.linalg as sla
    return np.sort(sla.eigsh(H, k=nroots, which="SA")[0])


# ---------------------------------------------------------------------------
# Block basis vectors of an MPS in Fock space (pins for the block algebra)
# ---------------------------------------------------------------------------

def left_block_vectors(mps, m: int):
    """{bond-m sector index: (4^m x d) basis of sites 1..m} from A[1..m]."""
    V = {0: np.ones((1, 1))}
    for k in range(1, m + 1):
        new = {}
        for (il, n, ir), blk in mps.sites[k].items():
            if il not in V:
                continue
            e = np.zeros((4, 1))
            e[n, 0] = 1.0
            contrib = np.kron(V[il], e) @ blk
            new[ir] = new.get(ir, 0) + contrib
        V = new
    return V


def right_block_vectors(mps, m: int):
    """{bond-m sector index: (4^(K-m) x d) basis of sites m+1..K}."""
    K = mps.K
    W = {0: np.ones((1, 1))}
    for k in range(K, m, -1):
        new = {}
        for (il, n, ir), blk in mps.sites[k].items():
            if ir not in W:
                continue
            e = np.zeros((4, 1))
            e[n, 0] = 1.0
            contrib = np.kron(e, W[ir]) @ blk.T
            new[il] = new.get(il, 0) + contrib
        W = new
    return W
