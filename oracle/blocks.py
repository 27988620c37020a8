"""Block-sparse operators, blocking and renormalisation (test infrastructure).

* ``Basis``: symmetry sectors (N, 2Sz) of a block, each a dense range of states
  (Abelian symmetry => block sparsity, Sec. 2.2).
* ``Op``: an operator with a definite change of quantum numbers, stored as one
  dense block per ket sector.
* ``BlockOps``: the operator set of Eq. (qops) for one block X:
  a+_p (p in X), A_pq = a+p a+q and B_ps = a+p a_s (p, q, s in X, all pairs for
  B), S_p (p not in X) and H^X.  P_pq and Q_ps are formed from A and B by their
  definitions whenever they are needed (``P`` / ``Q`` below).
* ``site_block``: the exact operators of one spatial orbital, from the 4x4
  creation matrices, by definition.
* ``block_product``: the operators of the union X.Y of two blocks (X left of Y
  in Jordan-Wigner order) from those of X and Y.  The formulas come from
  splitting each defining sum by which block every index lies in and moving
  operators of X to the left (sign -1 per transposition of odd operators);
  a product O^X O^Y acts on |x y> as (-1)^{par(O^Y) n(x)} O^X|x> O^Y|y>,
  which is the factor zeta of Eqs. (Sigma) and (Renorm).
* ``left_projector`` / ``right_projector`` / ``project_block``: Eq. (Renorm),
  O_new = A^+ O A with O the exact operator of the enlarged block.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import SITE_CREATORS

SITE_QN = [(0, 0), (1, -1), (1, 1), (2, 0)]


class Basis:
    def __init__(self, qns, dims):
        self.qn = [tuple(int(x) for x in q) for q in qns]
        self.dim = [int(d) for d in dims]
        self.index = {q: i for i, q in enumerate(self.qn)}

    def n(self, i):
        return self.qn[i][0]

    @property
    def size(self):
        return sum(self.dim)

    def offsets(self):
        off, o = [], 0
        for d in self.dim:
            off.append(o)
            o += d
        return off


SITE_BASIS = Basis(SITE_QN, [1, 1, 1, 1])


class Op:
    """Operator with quantum-number change ``dq`` = (dN, d2Sz); ``blocks[i]`` is
    the dense (dim_out x dim_in) block acting on ket sector i."""

    def __init__(self, basis, dq, blocks=None):
        self.basis = basis
        self.dq = (int(dq[0]), int(dq[1]))
        self.blocks = {} if blocks is None else blocks

    @property
    def parity(self):
        return self.dq[0] & 1

    def out(self, i):
        q = self.basis.qn[i]
        return self.basis.index.get((q[0] + self.dq[0], q[1] + self.dq[1]))

    @staticmethod
    def zero(basis, dq):
        return Op(basis, dq, {})

    @staticmethod
    def identity(basis):
        return Op(basis, (0, 0), {i: np.eye(d) for i, d in enumerate(basis.dim)})

    def copy(self):
        return Op(self.basis, self.dq, {i: b.copy() for i, b in self.blocks.items()})

    @property
    def T(self):
        blocks = {}
        for i, b in self.blocks.items():
            blocks[self.out(i)] = b.T.copy()
        return Op(self.basis, (-self.dq[0], -self.dq[1]), blocks)

    def scaled(self, c):
        return Op(self.basis, self.dq, {i: c * b for i, b in self.blocks.items()})

    def iadd(self, other, c=1.0):
        """self += c * other (same basis and dq)."""
        if other is None or c == 0.0:
            return self
        assert other.dq == self.dq, (other.dq, self.dq)
        for i, b in other.blocks.items():
            if i in self.blocks:
                self.blocks[i] = self.blocks[i] + c * b
            else:
                self.blocks[i] = c * b
        return self

    def __matmul__(self, other):
        """Operator product self * other."""
        dq = (self.dq[0] + other.dq[0], self.dq[1] + other.dq[1])
        blocks = {}
        for i, b in other.blocks.items():
            j = other.out(i)
            if j in self.blocks:
                blocks[i] = self.blocks[j] @ b
        return Op(self.basis, dq, blocks)

    def dense(self):
        off = self.basis.offsets()
        n = self.basis.size
        M = np.zeros((n, n))
        for i, b in self.blocks.items():
            j = self.out(i)
            M[off[j]:off[j] + b.shape[0], off[i]:off[i] + b.shape[1]] = b
        return M

    def diag(self):
        """Diagonal as {sector: vector} (only for dq = 0)."""
        assert self.dq == (0, 0)
        return {i: np.diag(b).copy() for i, b in self.blocks.items()}


# ---------------------------------------------------------------------------
# Operator set of one block
# ---------------------------------------------------------------------------

class BlockOps:
    """Operators of Eq. (qops) for one block; ``orbs`` are its spin orbitals."""

    def __init__(self, basis, orbs, n_so, hso, w):
        self.basis = basis
        self.orbs = sorted(orbs)
        self.others = [p for p in range(n_so) if p not in set(orbs)]
        self.hso, self.w = hso, w
        self.C, self.A, self.B, self.S = {}, {}, {}, {}
        self.H = None

    def I(self):
        return Op.identity(self.basis)

    def lincomb(self, kind: str, coefs: dict, dq) -> Op:
        """sum_k coefs[k] * ops[k] over the ``kind`` ('A' or 'B') operators with
        change ``dq`` (a contraction over a stacked array per ket sector)."""
        fam = self._family(kind, dq)
        out = Op.zero(self.basis, dq)
        if fam is None:
            return out
        keys, stacks = fam
        c = np.array([coefs.get(k, 0.0) for k in keys])
        if not np.any(c):
            return out
        for i, st in stacks.items():
            out.blocks[i] = np.tensordot(c, st, axes=1)
        return out

    def _family(self, kind, dq):
        cache = self.__dict__.setdefault("_fam_cache", {})
        if (kind, dq) not in cache:
            ops = self.A if kind == "A" else self.B
            keys = [k for k, o in ops.items() if o.dq == dq]
            if not keys:
                cache[(kind, dq)] = None
            else:
                sectors = sorted({i for k in keys for i in ops[k].blocks})
                stacks = {}
                for i in sectors:
                    j = ops[keys[0]].out(i)
                    shape = (self.basis.dim[j], self.basis.dim[i])
                    stacks[i] = np.stack([ops[k].blocks.get(i, np.zeros(shape)) for k in keys])
                cache[(kind, dq)] = (keys, stacks)
        return cache[(kind, dq)]

    def P(self, p, q):
        """P_pq = sum_{s<r in X} <pq||sr> a_r a_s = (sum_{s<r} w_pqsr A_sr)^T."""
        dqA = (2, _spin(p) + _spin(q))
        coefs = {(s, r): self.w[p, q, s, r] for (s, r) in self.A}
        return self.lincomb("A", coefs, dqA).T

    def Q(self, p, s):
        """Q_ps = sum_{q,r in X} <pq||sr> a+_q a_r = sum w_pqsr B_qr."""
        dq = (0, _spin(s) - _spin(p))
        coefs = {(q, r): self.w[p, q, s, r] for (q, r) in self.B}
        return self.lincomb("B", coefs, dq)


def _spin(p):
    return 1 if p % 2 == 0 else -1


def exact_block(basis, creators, orbs, n_so, hso, w):
    """All operators of a block whose creators ``creators[p]`` are exact
    (a full Fock space), built directly from the definitions of Eq. (qops)."""
    X = BlockOps(basis, orbs, n_so, hso, w)
    cd = {p: creators[p] for p in X.orbs}
    an = {p: c.T for p, c in cd.items()}
    for p in X.orbs:
        X.C[p] = cd[p]
    for i, p in enumerate(X.orbs):
        for q in X.orbs[i + 1:]:
            X.A[(p, q)] = cd[p] @ cd[q]
    for p in X.orbs:
        for s in X.orbs:
            X.B[(p, s)] = cd[p] @ an[s]
    for p in X.others:
        S = Op.zero(basis, (-1, -_spin(p)))
        for q in X.orbs:
            if hso[p, q] != 0.0:
                S.iadd(an[q], 0.5 * hso[p, q])
        for q in X.orbs:
            for i, s in enumerate(X.orbs):
                for r in X.orbs[i + 1:]:
                    c = w[p, q, s, r]
                    if c != 0.0:
                        S.iadd(cd[q] @ an[r] @ an[s], c)
        X.S[p] = S
    H = Op.zero(basis, (0, 0))
    for p in X.orbs:
        for q in X.orbs:
            if hso[p, q] != 0.0:
                H.iadd(cd[p] @ an[q], hso[p, q])
    for i, p in enumerate(X.orbs):
        for q in X.orbs[i + 1:]:
            for j, s in enumerate(X.orbs):
                for r in X.orbs[j + 1:]:
                    c = w[p, q, s, r]
                    if c != 0.0:
                        H.iadd(cd[p] @ cd[q] @ an[r] @ an[s], c)
    X.H = H
    return X


def site_block(k, n_so, hso, w):
    """Exact operators of spatial orbital k (0-based), local basis {vac,b,a,ab}."""
    creators = {}
    for s in (0, 1):
        M = SITE_CREATORS[s]
        blocks = {}
        for i in range(4):
            j = int(np.argmax(np.abs(M[:, i])))
            if M[j, i] != 0.0:
                blocks[i] = np.array([[M[j, i]]])
        creators[2 * k + s] = Op(SITE_BASIS, (1, 1 if s == 0 else -1), blocks)
    return exact_block(SITE_BASIS, creators, [2 * k, 2 * k + 1], n_so, hso, w)


# ---------------------------------------------------------------------------
# Product of two blocks
# ---------------------------------------------------------------------------

class ProductBasis(Basis):
    """Basis |x y> of X.Y; each sector lists its components (ix, iy) in order."""

    def __init__(self, BX, BY):
        comps = {}
        for ix, qx in enumerate(BX.qn):
            for iy, qy in enumerate(BY.qn):
                q = (qx[0] + qy[0], qx[1] + qy[1])
                comps.setdefault(q, []).append((ix, iy))
        qns = sorted(comps)
        self.BX, self.BY = BX, BY
        self.comps = [comps[q] for q in qns]
        self.comp_off = []
        dims = []
        for cl in self.comps:
            offs, o = {}, 0
            for (ix, iy) in cl:
                offs[(ix, iy)] = o
                o += BX.dim[ix] * BY.dim[iy]
            self.comp_off.append(offs)
            dims.append(o)
        super().__init__(qns, dims)

    def locate(self, ix, iy):
        q = (self.BX.qn[ix][0] + self.BY.qn[iy][0], self.BX.qn[ix][1] + self.BY.qn[iy][1])
        i = self.index[q]
        return i, self.comp_off[i][(ix, iy)]


def kron(PB, OX, OY):
    """(O^X O^Y)|x y> = (-1)^{par(O^Y) n(x)} O^X|x> O^Y|y>; None = identity."""
    dqx = (0, 0) if OX is None else OX.dq
    dqy = (0, 0) if OY is None else OY.dq
    pary = 0 if OY is None else OY.parity
    out = Op(PB, (dqx[0] + dqy[0], dqx[1] + dqy[1]), {})
    for i, cl in enumerate(PB.comps):
        for (ix, iy) in cl:
            if OX is None:
                jx, bx = ix, None
            else:
                if ix not in OX.blocks:
                    continue
                jx, bx = OX.out(ix), OX.blocks[ix]
            if OY is None:
                jy, by = iy, None
            else:
                if iy not in OY.blocks:
                    continue
                jy, by = OY.out(iy), OY.blocks[iy]
            sign = -1.0 if (pary and (PB.BX.n(ix) & 1)) else 1.0
            bx = np.eye(PB.BX.dim[ix]) if bx is None else bx
            by = np.eye(PB.BY.dim[iy]) if by is None else by
            blk = sign * np.kron(bx, by)
            j, ro = PB.locate(jx, jy)
            _, co = PB.locate(ix, iy)
            if i not in out.blocks:
                out.blocks[i] = np.zeros((PB.dim[j], PB.dim[i]))
            out.blocks[i][ro:ro + blk.shape[0], co:co + blk.shape[1]] += blk
    return out


def block_product(X: BlockOps, Y: BlockOps, normal: str | None = None) -> BlockOps:
    """Operators of the union block Z = X.Y (every orbital of X precedes Y)."""
    assert not X.orbs or not Y.orbs or max(X.orbs) < min(Y.orbs)
    PB = ProductBasis(X.basis, Y.basis)
    n_so = X.hso.shape[0]
    w, hso = X.w, X.hso
    Z = BlockOps(PB, X.orbs + Y.orbs, n_so, hso, w)
    for p in X.orbs:
        Z.C[p] = kron(PB, X.C[p], None)
    for p in Y.orbs:
        Z.C[p] = kron(PB, None, Y.C[p])
    for (p, q), A in X.A.items():
        Z.A[(p, q)] = kron(PB, A, None)
    for (p, q), A in Y.A.items():
        Z.A[(p, q)] = kron(PB, None, A)
    for p in X.orbs:
        for q in Y.orbs:
            Z.A[(p, q)] = kron(PB, X.C[p], Y.C[q])
    for (p, s), B in X.B.items():
        Z.B[(p, s)] = kron(PB, B, None)
    for (p, s), B in Y.B.items():
        Z.B[(p, s)] = kron(PB, None, B)
    for p in X.orbs:
        for s in Y.orbs:
            Z.B[(p, s)] = kron(PB, X.C[p], Y.C[s].T)             # a+p^X a_s^Y
            Z.B[(s, p)] = kron(PB, X.C[p].T, Y.C[s]).scaled(-1.0)  # a+s^Y a_p^X = -a_p^X a+s^Y
    # S_p for p outside Z
    for p in Z.others:
        S = kron(PB, X.S[p], None)
        S.iadd(kron(PB, None, Y.S[p]))
        for q in X.orbs:
            S.iadd(kron(PB, X.C[q], Y.P(p, q)))
        for q in Y.orbs:
            S.iadd(kron(PB, X.P(p, q), Y.C[q]))
        for r in Y.orbs:
            S.iadd(kron(PB, X.Q(p, r), Y.C[r].T))
        for s in X.orbs:
            S.iadd(kron(PB, X.C[s].T, Y.Q(p, s)))
        Z.S[p] = S
    Z.H = two_block_hamiltonian(PB, X, Y, normal)
    return Z


def two_block_terms(X: BlockOps, Y: BlockOps, normal: str | None = None):
    """Yield (coef, O^X, O^Y) with H(X.Y) = sum coef * O^X O^Y (X-left products):
    H^X + H^Y + sum_{p in X}(a+p S^Y_p + h.c.) + sum_{p in Y}(a+p S^X_p + h.c.)
    + sum_{p<q}(A_pq P_pq + h.c.) + sum_{p,s} B_ps Q_ps, the normal operators
    on ``normal`` ('X' or 'Y'; default the block with fewer orbitals).
    Reordering: a+^Y S^X = -S^X a+^Y and (a+^X S^Y)^+ = -a^X (S^Y)^+.
    ``None`` stands for the identity."""
    if normal is None:
        normal = "X" if len(X.orbs) <= len(Y.orbs) else "Y"
    yield 1.0, X.H, None
    yield 1.0, None, Y.H
    for p in X.orbs:
        yield 1.0, X.C[p], Y.S[p]
        yield -1.0, X.C[p].T, Y.S[p].T
    for p in Y.orbs:
        yield -1.0, X.S[p], Y.C[p]
        yield 1.0, X.S[p].T, Y.C[p].T
    if normal == "X":
        for (p, q), A in X.A.items():
            P = Y.P(p, q)
            yield 1.0, A, P
            yield 1.0, A.T, P.T
        for (p, s), B in X.B.items():
            yield 1.0, B, Y.Q(p, s)
    else:
        for (p, q), A in Y.A.items():
            P = X.P(p, q)
            yield 1.0, P, A
            yield 1.0, P.T, A.T
        for (p, s), B in Y.B.items():
            yield 1.0, X.Q(p, s), B


def two_block_hamiltonian(PB, X: BlockOps, Y: BlockOps, normal: str | None = None) -> Op:
    """H of the union block X.Y as an operator on the product basis."""
    H = Op.zero(PB, (0, 0))
    for c, OX, OY in two_block_terms(X, Y, normal):
        H.iadd(kron(PB, OX, OY), c)
    return H


# ---------------------------------------------------------------------------
# Renormalisation, Eq. (Renorm)
# ---------------------------------------------------------------------------

def left_projector(PB: ProductBasis, site_blocks, new_basis: Basis):
    """U[ir] (dim of enlarged sector x d_r) from A[k][(il, n, ir)] (left block)."""
    U = {}
    for ir, q in enumerate(new_basis.qn):
        i = PB.index[q]
        M = np.zeros((PB.dim[i], new_basis.dim[ir]))
        for (il, n), off in PB.comp_off[i].items():
            blk = site_blocks.get((il, n, ir))
            if blk is not None:
                M[off:off + blk.shape[0]] = blk
        U[ir] = (i, M)
    return U


def right_projector(PB: ProductBasis, site_blocks, new_basis: Basis):
    """V[il] (enlarged sector dim x d_l) from A[k][(il, n, ir)] (right block)."""
    V = {}
    for il, q in enumerate(new_basis.qn):
        i = PB.index[q]
        M = np.zeros((PB.dim[i], new_basis.dim[il]))
        for (n, ir), off in PB.comp_off[i].items():
            blk = site_blocks.get((il, n, ir))
            if blk is not None:
                M[off:off + blk.shape[1]] = blk.T
        V[il] = (i, M)
    return V


def project(op: Op, U, new_basis: Basis) -> Op:
    """O_new[r', r] = sum A*[l'c', r'] O[l'c', lc] A[lc, r]  (Eq. Renorm)."""
    out = Op(new_basis, op.dq, {})
    enl_to_new = {i: ir for ir, (i, _) in U.items()}
    for ir, (i, M) in U.items():
        if i not in op.blocks:
            continue
        j = op.out(i)
        jr = enl_to_new.get(j)
        if jr is None:
            continue
        out.blocks[ir] = U[jr][1].T @ op.blocks[i] @ M
    return out


def project_block(Z: BlockOps, U, new_basis: Basis) -> BlockOps:
    R = BlockOps(new_basis, Z.orbs, Z.hso.shape[0], Z.hso, Z.w)
    R.C = {p: project(o, U, new_basis) for p, o in Z.C.items()}
    R.A = {k: project(o, U, new_basis) for k, o in Z.A.items()}
    R.B = {k: project(o, U, new_basis) for k, o in Z.B.items()}
    R.S = {p: project(o, U, new_basis) for p, o in Z.S.items()}
    R.H = project(Z.H, U, new_basis)
    return R


def vacuum_block(n_so, hso, w, qn=(0, 0)) -> BlockOps:
    """The empty block (one state, no orbitals): all S_p and H vanish."""
    B = BlockOps(Basis([qn], [1]), [], n_so, hso, w)
    for p in B.others:
        B.S[p] = Op.zero(B.basis, (-1, -_spin(p)))
    B.H = Op.zero(B.basis, (0, 0))
    return B
