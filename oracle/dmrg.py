"""Environments, Davidson, decimation and the two-dot sweep (test infrastructure).

* ``Oracle.left_block(m)`` / ``right_block(m)``: renormalised operators of sites
  1..m / m+1..K by repeated blocking with one site and projection, Eq. (Renorm).
* ``davidson``: block Davidson (Davidson 1975, cited in Sec. 2.1) with the
  diagonal preconditioner t_i = -r_i / (H_ii - theta), modified Gram-Schmidt
  applied twice, subspace <= 20 n_roots and restart to the Ritz vectors plus the
  last corrections; converged when every ||r|| <= tol.
* ``decimate``: SVD (one root) or state-averaged density matrix (several roots)
  per sector of the bond between the two sites, keep the D largest weights
  globally (ties broken by sector order, then index), discarded weight w.
* ``Oracle.sweep``: forward over bonds (1,2)..(K-2,K-1), then backward over
  (K-1,K)..(2,3); forward updates A[k], backward A[k+1] (Sec. 2.3).
"""
from __future__ import annotations

import numpy as np

from synthetic_inputs import MPS

from .blocks import (SITE_QN, Basis, block_product, left_projector, project_block,
                     right_projector, site_block, vacuum_block)
from .hamiltonian import spin_orbital_integrals
from .sigma import TwoSite, two_site_layout


class Oracle:
    def __init__(self, h, eri, N, twoS, mps: MPS):
        self.K, self.N, self.twoS = h.shape[0], N, twoS
        self.hso, self.w = spin_orbital_integrals(h, eri)
        self.n_so = 2 * self.K
        self.mps = mps
        self._left = {}    # m -> BlockOps of sites 1..m
        self._right = {}   # m -> BlockOps of sites m+1..K

    # -- environments ------------------------------------------------------
    def _bond_basis_left(self, b):
        secs = self.mps.bonds[b]
        return Basis([(s[0], s[1]) for s in secs], [s[2] for s in secs])

    def _bond_basis_right(self, b):
        secs = self.mps.bonds[b]
        return Basis([(self.N - s[0], self.twoS - s[1]) for s in secs], [s[2] for s in secs])

    def left_block(self, m):
        if m in self._left:
            return self._left[m]
        if m == 0:
            X = vacuum_block(self.n_so, self.hso, self.w)
        else:
            prev = self.left_block(m - 1)
            Z = block_product(prev, site_block(m - 1, self.n_so, self.hso, self.w))
            nb = self._bond_basis_left(m)
            X = project_block(Z, left_projector(Z.basis, self.mps.sites[m], nb), nb)
        self._left[m] = X
        return X

    def right_block(self, m):
        if m in self._right:
            return self._right[m]
        if m == self.K:
            Y = vacuum_block(self.n_so, self.hso, self.w)
        else:
            nxt = self.right_block(m + 1)
            Z = block_product(site_block(m, self.n_so, self.hso, self.w), nxt)
            nb = self._bond_basis_right(m)
            Y = project_block(Z, right_projector(Z.basis, self.mps.sites[m + 1], nb), nb)
        self._right[m] = Y
        return Y

    def two_site(self, k) -> TwoSite:
        """Two-site problem at bond (k, k+1): L = sites 1..k-1, R = k+2..K."""
        return TwoSite(self.left_block(k - 1), self.right_block(k + 1), k, self.N, self.twoS)

    # -- one bond --------------------------------------------------------
    def optimise_bond(self, k, guess, n_roots=1, tol=1e-6, max_iter=200):
        ts = self.two_site(k)
        diag = ts.hdiag()
        X0 = np.atleast_2d(guess)
        theta, X, iters = davidson(lambda v: ts.sigma(v), diag, X0, n_roots, tol, max_iter)
        return ts, theta, X, iters

    def sweep(self, n_sweeps, D, n_roots=1, guess=None, tol=1e-6, max_iter=200,
              D_schedule=None):
        """Two-dot sweeps starting at bond (1,2).  Returns (energies, discarded,
        bond_energies): per sweep the lowest-root energy at its last bond and the
        largest discarded weight, and the lowest-root energy of every bond."""
        assert self.mps.center == 1
        K = self.K
        if guess is None:
            from synthetic_inputs import random_vector
            guess = random_vector(self.two_site(1).dim, seed=1, nvec=n_roots)
        psi = np.atleast_2d(guess)
        energies, discarded, bond_energies = [], [], []
        for sw in range(n_sweeps):
            Dk = D if D_schedule is None else D_schedule[sw]
            wmax = 0.0
            plan = [(k, True) for k in range(1, K - 1)] + [(k, False) for k in range(K - 1, 1, -1)]
            for k, forward in plan:
                ts, theta, X, _ = self.optimise_bond(k, psi, n_roots, tol, max_iter)
                bond_energies.append(theta[0])
                w, psi = self.decimate_and_move(ts, k, X, Dk, forward)
                wmax = max(wmax, w)
            energies.append(bond_energies[-1])
            discarded.append(wmax)
        return np.array(energies), np.array(discarded), np.array(bond_energies)

    # -- decimation --------------------------------------------------------
    def decimate_and_move(self, ts: TwoSite, k, X, D, forward):
        """Truncate the bond between sites k and k+1, update A[k] (forward) or
        A[k+1] (backward), move the centre and return (w, guesses for the next
        bond): the centre tensor C = U^T M (or M V) contracted with the
        neighbouring site tensor."""
        mps = self.mps
        groups, kept, w = decimate(ts.layout, X, [b[0:2] for b in mps.bonds[k - 1]],
                                   [b[0:2] for b in mps.bonds[k + 1]], D, forward)
        new_index = {q: i for i, (q, _, _) in enumerate(kept)}
        blocks = {}
        if forward:
            for q, U, rows in kept:
                for (il, c1, off, dl) in rows:
                    blocks[(il, c1, new_index[q])] = U[off:off + dl].copy()
        else:
            for q, V, cols in kept:
                for (c2, ir, off, dr) in cols:
                    blocks[(new_index[q], c2, ir)] = V[off:off + dr].T.copy()
        mps.bonds[k] = [(q[0], q[1], U.shape[1]) for q, U, _ in kept]
        mps.sites[k if forward else k + 1] = blocks
        nvec = X.shape[0]
        if forward:
            self._left = {m: v for m, v in self._left.items() if m < k}
            self._right = {m: v for m, v in self._right.items() if m >= k}
            mps.center = k + 1
            nxt = mps.sites[k + 2]
            layout, dim = two_site_layout([b[0:2] for b in mps.bonds[k]], [b[2] for b in mps.bonds[k]],
                                          [b[0:2] for b in mps.bonds[k + 2]], [b[2] for b in mps.bonds[k + 2]])
            guesses = np.zeros((nvec, dim))
            for v in range(nvec):
                C = {}
                for q, U, _ in kept:
                    Cm = U.T @ groups[q]["mats"][v]
                    for (c2, ir, off, dr) in groups[q]["cols"]:
                        C[(new_index[q], c2, ir)] = Cm[:, off:off + dr]
                for (il, c1, c2, ir, off, dl, dr) in layout:
                    acc = np.zeros((dl, dr))
                    for (a, c, r), blk in C.items():
                        if a == il and c == c1 and (r, c2, ir) in nxt:
                            acc += blk @ nxt[(r, c2, ir)]
                    guesses[v, off:off + dl * dr] = acc.ravel()
        else:
            self._left = {m: v for m, v in self._left.items() if m <= k}
            self._right = {m: v for m, v in self._right.items() if m > k}
            mps.center = k - 1
            prv = mps.sites[k - 1]
            layout, dim = two_site_layout([b[0:2] for b in mps.bonds[k - 2]], [b[2] for b in mps.bonds[k - 2]],
                                          [b[0:2] for b in mps.bonds[k]], [b[2] for b in mps.bonds[k]])
            guesses = np.zeros((nvec, dim))
            for v in range(nvec):
                C = {}
                for q, V, _ in kept:
                    Cm = groups[q]["mats"][v] @ V
                    for (il, c1, off, dl) in groups[q]["rows"]:
                        C[(il, c1, new_index[q])] = Cm[off:off + dl, :]
                for (il, c0, c1, ir, off, dl, dr) in layout:
                    acc = np.zeros((dl, dr))
                    for (l, c, r), blk in C.items():
                        if c == c1 and r == ir and (il, c0, l) in prv:
                            acc += prv[(il, c0, l)] @ blk
                    guesses[v, off:off + dl * dr] = acc.ravel()
        return w, guesses


def decimate(layout, X, left_labels, right_labels, D, forward, cutoff=1e-14):
    """Group the two-site vectors X (n_roots x dim) by the label q of the bond
    between the two sites, M_q[(il c1), (c2 ir)]; for one root take the SVD of
    every M_q and keep the D largest singular values s > cutoff (weights s^2);
    for several roots the eigenvalues of the state-averaged density matrix,
    kept above cutoff^2.  Ties break by sector order, then index."""
    groups = {}
    for (il, c1, c2, ir, off, dl, dr) in layout:
        ql = left_labels[il]
        q = (ql[0] + SITE_QN[c1][0], ql[1] + SITE_QN[c1][1])
        g = groups.setdefault(q, {"rows": [], "cols": [], "rowoff": {}, "coloff": {}, "blocks": []})
        if (il, c1) not in g["rowoff"]:
            g["rowoff"][(il, c1)] = sum(r[3] for r in g["rows"])
            g["rows"].append((il, c1, g["rowoff"][(il, c1)], dl))
        if (c2, ir) not in g["coloff"]:
            g["coloff"][(c2, ir)] = sum(c[3] for c in g["cols"])
            g["cols"].append((c2, ir, g["coloff"][(c2, ir)], dr))
        g["blocks"].append((il, c1, c2, ir, off, dl, dr))
    qs = sorted(groups)
    nvec = X.shape[0]
    cands = []  # (-weight, group order, index, q)
    decomp = {}
    for gi, q in enumerate(qs):
        g = groups[q]
        nr = sum(r[3] for r in g["rows"])
        nc = sum(c[3] for c in g["cols"])
        mats = []
        for v in range(nvec):
            M = np.zeros((nr, nc))
            for (il, c1, c2, ir, off, dl, dr) in g["blocks"]:
                ro, co = g["rowoff"][(il, c1)], g["coloff"][(c2, ir)]
                M[ro:ro + dl, co:co + dr] = X[v, off:off + dl * dr].reshape(dl, dr)
            mats.append(M)
        g["mats"] = mats
        if nvec == 1:
            # one root: singular values of M_q (their squares are the weights);
            # left vectors for the forward move, right vectors backward
            U, s, Vt = np.linalg.svd(mats[0], full_matrices=False)
            lam, vec = s * s, (U if forward else Vt.T)
        else:
            # several roots: state-averaged density matrix, equal weights
            if forward:
                rho = sum(M @ M.T for M in mats) / nvec
            else:
                rho = sum(M.T @ M for M in mats) / nvec
            lam, vec = np.linalg.eigh(rho)
        order = np.argsort(-lam, kind="stable")
        lam, vec = lam[order], vec[:, order]
        decomp[q] = (lam, vec)
        for i, l in enumerate(lam):
            cands.append((-l, gi, i, q))
    cands.sort(key=lambda t: (t[0], t[1], t[2]))
    keep = {}
    w = 0.0
    nkept = 0
    for (negl, gi, i, q) in cands:
        lam = -negl
        if nkept < D and lam > cutoff ** 2:
            keep.setdefault(q, []).append(i)
            nkept += 1
        else:
            w += max(lam, 0.0)
    kept = []
    for q in qs:
        if q not in keep:
            continue
        idx = sorted(keep[q])
        vec = decomp[q][1][:, idx]
        kept.append((q, vec, groups[q]["rows"] if forward else groups[q]["cols"]))
    return groups, kept, w


def davidson(matvec, diag, X0, n_roots=1, tol=1e-6, max_iter=200, max_space=None):
    """Lowest ``n_roots`` eigenpairs of a symmetric operator given by ``matvec``."""
    n = diag.size
    max_space = max_space or 20 * n_roots
    V = np.zeros((0, n))
    W = np.zeros((0, n))
    new = np.array(X0, dtype=float).reshape(-1, n)
    it = 0
    while True:
        # orthonormalise the new directions against V (MGS, twice)
        add = []
        for t in new:
            for _ in range(2):
                for v in list(V) + add:
                    t = t - (v @ t) * v
            nt = np.linalg.norm(t)
            if nt > 1e-10:
                add.append(t / nt)
        if add:
            A = np.array(add)
            V = np.vstack([V, A])
            W = np.vstack([W, np.array([matvec(a) for a in A])])
        G = V @ W.T
        G = 0.5 * (G + G.T)
        theta, Y = np.linalg.eigh(G)
        theta, Y = theta[:n_roots], Y[:, :n_roots]
        X = Y.T @ V
        R = Y.T @ W - theta[:, None] * X
        rnorm = np.linalg.norm(R, axis=1)
        it += 1
        if np.all(rnorm <= tol) or it >= max_iter or not add:
            return theta, X, it
        T = []
        for i in range(n_roots):
            den = diag - theta[i]
            den = np.where(np.abs(den) < 1e-8, np.where(den < 0, -1e-8, 1e-8), den)
            T.append(-R[i] / den)
        new = np.array(T)
        if V.shape[0] + n_roots > max_space:
            V, W = X.copy(), Y.T @ W
            # re-orthonormalise the restarted Ritz basis
            Qm, Rm = np.linalg.qr(V.T)
            V = Qm.T
            W = np.linalg.solve(Rm.T, W) if Rm.shape[0] == Rm.shape[1] else W
