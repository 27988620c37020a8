"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only *generates* inputs: one- and two-electron integrals (as
Cholesky vectors), the symmetry-sector dimensions of a matrix product state,
random MPS site tensors, random vectors, and the binary MPS file format that
both sides read.  It contains none of the DMRG arithmetic (no operators, no
blocking, no sigma product, no eigensolver).

Integral recipe (a synthetic stand-in for the P-cluster FCIDUMP, whose shape
K=73 orbitals / N=114 electrons the largest workload reuses):

* ``h`` is symmetric, ``h[p, p] = linspace(h_min, 0, K)``, off-diagonal
  ``h[p, q] ~ N(0, (0.1 * exp(-|p-q|/ell))**2)`` (0.1*exp(..) is the standard
  deviation), drawn for the upper triangle in row-major order and mirrored;
* ``L[X, p, q] ~ N(0, (0.15 * exp(-|p-q|/ell))**2)`` symmetric in (p, q),
  drawn X-major over the upper triangle including the diagonal, row-major;
* the chemist-notation integrals are ``(pq|rs) = sum_X L[X,p,q] L[X,r,s]``
  (formed by each consumer, not here), which is 8-fold symmetric and PSD.

Random numbers come from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass, field

import numpy as np

# Local basis of one spatial orbital, in the order {vac, beta, alpha, alpha-beta}
# (paper Sec. 2.1, after Eq. MPS): index n = 2*n_alpha + n_beta.
SITE_QN = [(0, 0), (1, -1), (1, 1), (2, 0)]  # (particle number, 2*Sz)


def make_integrals(K: int, n_chol: int, ell: float = 3.0, h_min: float = -4.0,
                   seed: int = 0):
    """Return ``(h, L)``: h is (K, K) symmetric, L is (n_chol, K, K) symmetric."""
    rng = np.random.default_rng(seed)
    h = np.zeros((K, K))
    h[np.diag_indices(K)] = np.linspace(h_min, 0.0, K)
    iu, ju = np.triu_indices(K, 1)          # row-major upper triangle, i < j
    z = rng.standard_normal(iu.size)
    h[iu, ju] = z * 0.1 * np.exp(-np.abs(iu - ju) / ell)
    h[ju, iu] = h[iu, ju]
    L = np.zeros((n_chol, K, K))
    il, jl = np.triu_indices(K, 0)          # row-major upper triangle incl. diagonal
    scale = 0.15 * np.exp(-np.abs(il - jl) / ell)
    for x in range(n_chol):
        z = rng.standard_normal(il.size)
        L[x, il, jl] = z * scale
        L[x, jl, il] = L[x, il, jl]
    return h, L


# ---------------------------------------------------------------------------
# Sector dimensions of the MPS bonds
# ---------------------------------------------------------------------------

def _full_dim(nsites: int, na: int, nb: int) -> int:
    if na < 0 or nb < 0 or na > nsites or nb > nsites:
        return 0
    return math.comb(nsites, na) * math.comb(nsites, nb)


def _waterfill(weights, caps, budget):
    """Integer allocation of ``budget`` proportional to ``weights`` under caps."""
    n = len(weights)
    alloc = [0.0] * n
    active = [i for i in range(n) if caps[i] > 0 and weights[i] > 0]
    remaining = float(budget)
    while active and remaining > 1e-9:
        wsum = sum(weights[i] for i in active)
        capped = [i for i in active if alloc[i] + remaining * weights[i] / wsum >= caps[i]]
        if not capped:
            for i in active:
                alloc[i] += remaining * weights[i] / wsum
            remaining = 0.0
            break
        for i in capped:
            remaining -= caps[i] - alloc[i]
            alloc[i] = caps[i]
        active = [i for i in active if i not in capped]
    out = [min(caps[i], int(math.floor(alloc[i] + 1e-9))) for i in range(n)]
    # hand out the rounding remainder to the largest fractional parts
    left = min(budget, sum(caps)) - sum(out)
    order = sorted(range(n), key=lambda i: -(alloc[i] - math.floor(alloc[i] + 1e-9)))
    for i in order:
        if left <= 0:
            break
        if out[i] < caps[i] and weights[i] > 0:
            out[i] += 1
            left -= 1
    return out


def bond_sectors(K: int, N: int, twoS: int, D: int, split: str = "proportional",
                 width_n: float | None = None, width_s: float | None = None):
    """Sector list of every bond b = 0..K as ``[(N_L, 2Sz_L, dim), ...]``.

    Bond b separates sites 1..b (left) from b+1..K (right); the label is the
    quantum number of the left part.  ``split='proportional'`` shares D in
    proportion to the Schmidt-rank bound of each sector; ``split='gaussian'``
    shares it with a Gaussian in (N_L - N*b/K, 2Sz_L) (the "synthetic split").
    Dimensions are then made consistent so that left- and right-isometric
    site tensors exist.
    """
    Na, Nb = (N + twoS) // 2, (N - twoS) // 2
    assert Na + Nb == N and Na - Nb == twoS and 0 <= Na <= K and 0 <= Nb <= K
    bonds = []
    for b in range(K + 1):
        secs = []
        for na in range(0, min(b, Na) + 1):
            for nb in range(0, min(b, Nb) + 1):
                dl = _full_dim(b, na, nb)
                dr = _full_dim(K - b, Na - na, Nb - nb)
                cap = min(dl, dr)
                if cap > 0:
                    secs.append([na + nb, na - nb, cap])
        if split == "proportional":
            w = [float(s[2]) for s in secs]
        elif split == "gaussian":
            wn = width_n if width_n is not None else 2.0
            ws = width_s if width_s is not None else 2.0
            n0 = N * b / K
            w = [math.exp(-0.5 * ((s[0] - n0) / wn) ** 2 - 0.5 * (s[1] / ws) ** 2) for s in secs]
        else:
            raise ValueError(split)
        caps = [s[2] for s in secs]
        dims = _waterfill(w, caps, D)
        for s, d in zip(secs, dims):
            s[2] = d
        bonds.append(secs)
    # consistency: d_b(q) <= sum_n d_{b-1}(q - n) and d_b(q) <= sum_n d_{b+1}(q + n)
    for _ in range(4 * K + 4):
        changed = False
        for b in range(1, K + 1):
            prev = {(s[0], s[1]): s[2] for s in bonds[b - 1]}
            for s in bonds[b]:
                lim = sum(prev.get((s[0] - dn, s[1] - ds), 0) for dn, ds in SITE_QN)
                if s[2] > lim:
                    s[2] = lim
                    changed = True
        for b in range(K - 1, -1, -1):
            nxt = {(s[0], s[1]): s[2] for s in bonds[b + 1]}
            for s in bonds[b]:
                lim = sum(nxt.get((s[0] + dn, s[1] + ds), 0) for dn, ds in SITE_QN)
                if s[2] > lim:
                    s[2] = lim
                    changed = True
        if not changed:
            break
    return [[tuple(s) for s in secs if s[2] > 0] for secs in bonds]


# ---------------------------------------------------------------------------
# Random MPS and the binary MPS file format
# ---------------------------------------------------------------------------

@dataclass
class MPS:
    """Block-sparse MPS.

    ``bonds[b]`` is the sector list of bond b (b = 0..K).  ``sites[k]`` (k = 1..K,
    index 0 unused) maps ``(il, n, ir)`` to a dense ``d_l x d_r`` block, where il
    indexes bonds[k-1], n is the local state and ir indexes bonds[k].
    Sites ``< center`` are left-orthonormal, sites ``> center + 1`` are
    right-orthonormal; the two-site centre (center, center+1) is arbitrary.
    """
    K: int
    N: int
    twoS: int
    center: int
    bonds: list
    sites: list = field(default_factory=list)

    def block_keys(self, k: int):
        """Canonical block order of site k: il, then n, then the matching ir."""
        left, right = self.bonds[k - 1], self.bonds[k]
        ridx = {(s[0], s[1]): i for i, s in enumerate(right)}
        keys = []
        for il, (nl, sl, _) in enumerate(left):
            for n, (dn, ds) in enumerate(SITE_QN):
                ir = ridx.get((nl + dn, sl + ds))
                if ir is not None:
                    keys.append((il, n, ir))
        return keys


def random_mps(K: int, N: int, twoS: int, bonds, center: int = 1, seed: int = 2) -> MPS:
    """Random MPS with left-isometries left of ``center`` and right-isometries
    right of ``center + 1`` (orthonormalised per sector by QR)."""
    rng = np.random.default_rng(seed)
    mps = MPS(K, N, twoS, center, bonds, [None] * (K + 1))
    for k in range(1, K + 1):
        blocks = {}
        for key in mps.block_keys(k):
            il, n, ir = key
            blocks[key] = rng.standard_normal((bonds[k - 1][il][2], bonds[k][ir][2]))
        mps.sites[k] = blocks
    for k in range(1, K + 1):
        blocks = mps.sites[k]
        if k < center:  # left isometry: columns orthonormal over rows (il, n)
            for ir in range(len(bonds[k])):
                keys = [key for key in blocks if key[2] == ir]
                M = np.vstack([blocks[key] for key in keys])
                Q, _ = np.linalg.qr(M)
                row = 0
                for key in keys:
                    d = blocks[key].shape[0]
                    blocks[key] = np.ascontiguousarray(Q[row:row + d])
                    row += d
        elif k > center + 1:  # right isometry: rows orthonormal over cols (n, ir)
            for il in range(len(bonds[k - 1])):
                keys = [key for key in blocks if key[0] == il]
                M = np.hstack([blocks[key] for key in keys])
                Q, _ = np.linalg.qr(M.T)
                col = 0
                for key in keys:
                    d = blocks[key].shape[1]
                    blocks[key] = np.ascontiguousarray(Q[col:col + d].T)
                    col += d
    return mps


_MAGIC = b"DMRGMPS1"


def write_mps(path: str, mps: MPS) -> None:
    """Binary layout (little endian): magic, int32 K N twoS center; per bond
    int32 count then count x (int32 N_L, int32 2Sz_L, int32 dim); per site
    int32 nblocks then per block int32 (il, n, ir) and float64 data row-major."""
    with open(path, "wb") as f:
        f.write(_MAGIC)
        f.write(struct.pack("<4i", mps.K, mps.N, mps.twoS, mps.center))
        for secs in mps.bonds:
            f.write(struct.pack("<i", len(secs)))
            for s in secs:
                f.write(struct.pack("<3i", *s))
        for k in range(1, mps.K + 1):
            keys = mps.block_keys(k)
            f.write(struct.pack("<i", len(keys)))
            for key in keys:
                f.write(struct.pack("<3i", *key))
                f.write(np.ascontiguousarray(mps.sites[k][key], dtype="<f8").tobytes())


def read_mps(path: str) -> MPS:
    with open(path, "rb") as f:
        buf = f.read()
    assert buf[:8] == _MAGIC, "not an MPS file"
    off = 8
    K, N, twoS, center = struct.unpack_from("<4i", buf, off)
    off += 16
    bonds = []
    for _ in range(K + 1):
        (n,) = struct.unpack_from("<i", buf, off)
        off += 4
        secs = []
        for _ in range(n):
            secs.append(struct.unpack_from("<3i", buf, off))
            off += 12
        bonds.append(secs)
    mps = MPS(K, N, twoS, center, bonds, [None] * (K + 1))
    for k in range(1, K + 1):
        (nb,) = struct.unpack_from("<i", buf, off)
        off += 4
        blocks = {}
        for _ in range(nb):
            il, n, ir = struct.unpack_from("<3i", buf, off)
            off += 12
            dl, dr = bonds[k - 1][il][2], bonds[k][ir][2]
            blocks[(il, n, ir)] = np.frombuffer(buf, dtype="<f8", count=dl * dr,
                                                offset=off).reshape(dl, dr).copy()
            off += 8 * dl * dr
        mps.sites[k] = blocks
    return mps


def random_vector(n: int, seed: int = 1, nvec: int = 1) -> np.ndarray:
    """``nvec`` standard-normal vectors of length n, each normalised to 1."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((nvec, n))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v[0] if nvec == 1 else v


# Workload shapes (sizes of the paper-shaped synthetic problems).
WORKLOADS = {
    "k8_d64": dict(K=8, N=8, twoS=0, D=64, n_chol=32, ell=3.0, h_min=-4.0),
    "k36_d1000": dict(K=36, N=36, twoS=0, D=1000, n_chol=144, ell=3.0, h_min=-4.0),
    "k54_d2000": dict(K=54, N=54, twoS=0, D=2000, n_chol=216, ell=3.0, h_min=-4.0),
    "k73_d3000": dict(K=73, N=114, twoS=0, D=3000, n_chol=292, ell=8.0, h_min=-6.0),
}
