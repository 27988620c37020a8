"""Unit tests of the tcgen05 tensor-core engine (bf16 pieces, FP32 accumulation
in tensor memory) against numpy FP64: K-major and MN-major operands, ragged
M/N/K (tails inside a 128 x 128 tile and a 64-wide K stage), empty segment
lists, sign flips and epilogue scaling.

Error bound: |C - C_ref| <= c * u * (|A||B|) elementwise, with u = 2^-8 for
one bf16 piece and u = 2^-16 for two (hi + lo, products hi*hi + hi*lo +
lo*hi), c = 4 covering the FP32 accumulation of K <= 600 terms."""
import numpy as np
import pytest

from tests.helpers import cuda_torch, gpu_lib

pytestmark = pytest.mark.gpu


def _r8(x):
    return (x + 7) // 8 * 8


def _problem(rng, nblocks, sizes):
    A = rng.standard_normal(3_000_000)
    B = rng.standard_normal(3_000_000)
    blocks, ref, bound = [], [], []
    coff = aoff = boff = 0
    for bi in range(nblocks):
        m = int(rng.choice(sizes))
        n = int(rng.choice(sizes))
        nseg = int(rng.integers(0, 4))
        C = np.zeros((m, n))
        Bd = np.zeros((m, n))
        segs = []
        for _ in range(nseg):
            k = int(rng.choice([1, 8, 13, 64, 65, 200, 450]))
            at, bt = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            lda = _r8((m if at else k)) + 8 * int(rng.integers(0, 2))
            ldb = _r8((k if bt else n)) + 8 * int(rng.integers(0, 2))
            alpha = float(rng.choice([1.0, -1.0])) if nseg > 1 else float(rng.standard_normal())
            na = (k if at else m) * lda
            nb = (n if bt else k) * ldb
            Am = A[aoff:aoff + na].reshape(-1, lda)
            Bm = B[boff:boff + nb].reshape(-1, ldb)
            opA = Am[:k, :m].T if at else Am[:m, :k]
            opB = Bm[:n, :k].T if bt else Bm[:k, :n]
            C += alpha * opA @ opB
            Bd += abs(alpha) * np.abs(opA) @ np.abs(opB)
            segs.append((k, aoff, lda, at, boff, ldb, bt, alpha))
            aoff = _r8(aoff + na)
            boff = _r8(boff + nb)
        blocks.append((m, n, coff, segs))
        ref.append((coff, C))
        bound.append(Bd)
        coff += m * n
    assert aoff < A.size and boff < B.size
    return A, B, blocks, ref, bound, coff


@pytest.mark.parametrize("precision,u", [(1, 2.0 ** -16), (2, 2.0 ** -8), (3, 2.0 ** -19)])
@pytest.mark.parametrize("seed", [0, 1])
def test_tc_grouped_gemm_vs_fp64(precision, u, seed):
    torch = cuda_torch()
    g = gpu_lib()
    rng = np.random.default_rng(100 + seed)
    A, B, blocks, ref, bound, ctot = _problem(rng, 10, [1, 5, 64, 127, 128, 129, 300])
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((max(ctot, 1),), np.nan, dtype=torch.float64, device="cuda")
    g.grouped_gemm(precision, blocks, dA, dB, dC)
    C = dC.cpu().numpy()
    for (off, Cr), Bd, (m, n, _, _) in zip(ref, bound, blocks):
        got = C[off:off + m * n].reshape(m, n)
        assert np.all(np.isfinite(got))
        err = np.abs(got - Cr)
        assert np.all(err <= 4 * u * Bd + 1e-300), (err / (Bd + 1e-300)).max()


def test_tc_large_k_accumulation():
    """One 300 x 260 block summing 40 segments (K = 40 x 450): the whole term
    list of an output tile runs through one accumulator."""
    torch = cuda_torch()
    g = gpu_lib()
    rng = np.random.default_rng(7)
    m, n, k = 300, 260, 450
    segs, C, Bd = [], np.zeros((m, n)), np.zeros((m, n))
    A = rng.standard_normal(40 * m * _r8(k) + 8)
    B = rng.standard_normal(40 * n * _r8(k) + 8)
    for s in range(40):
        lda, ldb = _r8(k), _r8(k)
        ao, bo = s * m * lda, s * n * ldb
        Am = A[ao:ao + m * lda].reshape(m, lda)[:, :k]
        Bm = B[bo:bo + n * ldb].reshape(n, ldb)[:, :k]
        sg = 1.0 if s % 3 else -1.0
        C += sg * Am @ Bm.T
        Bd += np.abs(Am) @ np.abs(Bm.T)
        segs.append((k, ao, lda, 0, bo, ldb, 1, sg))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    g.grouped_gemm(1, [(m, n, 0, segs)], dA, dB, dC)
    got = dC.cpu().numpy().reshape(m, n)
    assert np.all(np.abs(got - C) <= 8 * 2.0 ** -16 * Bd)
