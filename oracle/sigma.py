"""Two-site sigma vector sigma = H psi, Eq. (Sigma), and diag(H_eff) (test infrastructure).

The superblock is split as S = L.C1 and E = C2.R.  The operators of S and E
are formed exactly from those of L, R and the two sites (``block_product``),
and H acting in the product space is the two-block sum of ``two_block_terms``;
each term O^S O^E acts on the wavefunction matrix Psi[(l c1), (c2 r)] as
(-1)^{par(O^E) n(l c1)} O^S Psi (O^E)^T.  This equals <l'c1'c2'r'|H|psi> because
every stored operator is the exact projection of its Fock-space operator.

Canonical layout of psi and sigma (also the layout of the C library): sectors
ordered by (left sector il, c1 = 0..3, c2 = 0..3), the right sector being the
one whose bond label is label(il) + q(c1) + q(c2); each block is d_l x d_r,
row-major.
"""
from __future__ import annotations

import numpy as np

from .blocks import SITE_QN, BlockOps, block_product, site_block, two_block_terms


def two_site_layout(left_labels, left_dims, right_labels, right_dims):
    """[(il, c1, c2, ir, offset, d_l, d_r)] in canonical order; labels are the
    (N_L, 2Sz_L) bond labels of the left and right bonds of the two sites."""
    ridx = {tuple(q): i for i, q in enumerate(right_labels)}
    out, off = [], 0
    for il, ql in enumerate(left_labels):
        for c1 in range(4):
            for c2 in range(4):
                q = (ql[0] + SITE_QN[c1][0] + SITE_QN[c2][0], ql[1] + SITE_QN[c1][1] + SITE_QN[c2][1])
                ir = ridx.get(q)
                if ir is None:
                    continue
                dl, dr = left_dims[il], right_dims[ir]
                out.append((il, c1, c2, ir, off, dl, dr))
                off += dl * dr
    return out, off


class TwoSite:
    """Two-site problem at bond (k, k+1) (1-based sites) from the left block L
    (sites 1..k-1) and right block R (sites k+2..K)."""

    def __init__(self, L: BlockOps, R: BlockOps, k: int, N: int, twoS: int):
        n_so = L.hso.shape[0]
        self.tot = (N, twoS)
        self.L, self.R = L, R
        self.S = block_product(L, site_block(k - 1, n_so, L.hso, L.w))
        self.E = block_product(site_block(k, n_so, L.hso, L.w), R)
        left_labels = L.basis.qn
        right_labels = [(N - q[0], twoS - q[1]) for q in R.basis.qn]
        self.layout, self.dim = two_site_layout(left_labels, L.basis.dim, right_labels, R.basis.dim)
        SB, EB = self.S.basis, self.E.basis
        # pair each S sector with the E sector completing the total quantum number
        self.pair = {}
        for iS, q in enumerate(SB.qn):
            iE = EB.index.get((N - q[0], twoS - q[1]))
            if iE is not None:
                self.pair[iS] = iE

    def to_se(self, psi):
        SB, EB = self.S.basis, self.E.basis
        X = {iS: np.zeros((SB.dim[iS], EB.dim[iE])) for iS, iE in self.pair.items()}
        for (il, c1, c2, ir, off, dl, dr) in self.layout:
            iS, ro = SB.locate(il, c1)
            iE, co = EB.locate(c2, ir)
            X[iS][ro:ro + dl, co:co + dr] = psi[off:off + dl * dr].reshape(dl, dr)
        return X

    def from_se(self, X):
        SB, EB = self.S.basis, self.E.basis
        out = np.zeros(self.dim)
        for (il, c1, c2, ir, off, dl, dr) in self.layout:
            iS, ro = SB.locate(il, c1)
            iE, co = EB.locate(c2, ir)
            if iS in X:
                out[off:off + dl * dr] = X[iS][ro:ro + dl, co:co + dr].ravel()
        return out

    def terms(self):
        """The two-block term list (materialised once; reused by every sigma)."""
        if not hasattr(self, "_terms"):
            self._terms = list(two_block_terms(self.S, self.E))
        return self._terms

    def sigma(self, psi, terms=None):
        """sigma = H psi for one vector in the canonical layout.  ``flops_last``
        receives the floating-point operations of the products and scaled sums
        this call performed (2mkn per matrix product, 2 per element summed)."""
        X = self.to_se(psi)
        SB = self.S.basis
        out = {}
        fl = 0
        for c, OS, OE in (self.terms() if terms is None else terms):
            pE = 0 if OE is None else OE.parity
            for iS, M in X.items():
                iE = self.pair[iS]
                if OS is None:
                    jS, A = iS, None
                elif iS in OS.blocks:
                    jS, A = OS.out(iS), OS.blocks[iS]
                else:
                    continue
                if OE is None:
                    B = None
                elif iE in OE.blocks:
                    B = OE.blocks[iE]
                else:
                    continue
                sign = -1.0 if (pE and (SB.n(iS) & 1)) else 1.0
                if A is not None:
                    fl += 2 * A.shape[0] * A.shape[1] * M.shape[1]
                T = M if A is None else A @ M
                if B is not None:
                    fl += 2 * T.shape[0] * T.shape[1] * B.shape[0]
                T = T if B is None else T @ B.T
                fl += 2 * T.size
                if jS in out:
                    out[jS] += (c * sign) * T
                else:
                    out[jS] = (c * sign) * T
        self.flops_last = fl
        return self.from_se(out)

    def hdiag(self):
        """Diagonal of H_eff: the terms whose two factors both conserve the
        quantum numbers contribute sign * diag(O^S) x diag(O^E)."""
        SB = self.S.basis
        out = {iS: np.zeros((SB.dim[iS], self.E.basis.dim[iE])) for iS, iE in self.pair.items()}
        for c, OS, OE in self.terms():
            dqS = (0, 0) if OS is None else OS.dq
            dqE = (0, 0) if OE is None else OE.dq
            if dqS != (0, 0) or dqE != (0, 0):
                continue
            pE = 0 if OE is None else OE.parity
            for iS, iE in self.pair.items():
                dS = np.ones(SB.dim[iS]) if OS is None else (
                    np.diag(OS.blocks[iS]) if iS in OS.blocks else None)
                dE = np.ones(self.E.basis.dim[iE]) if OE is None else (
                    np.diag(OE.blocks[iE]) if iE in OE.blocks else None)
                if dS is None or dE is None:
                    continue
                sign = -1.0 if (pE and (SB.n(iS) & 1)) else 1.0
                out[iS] += (c * sign) * np.outer(dS, dE)
        return self.from_se(out)
