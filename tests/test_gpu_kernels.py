"""Unit tests of the segmented grouped GEMM engine (the kernel behind every
sigma, renormalisation, intermediate and density-matrix product) against
numpy FP64 on random uneven work lists, including degenerate sizes."""
import numpy as np
import pytest

from tests.helpers import cuda_torch, gpu_lib

pytestmark = pytest.mark.gpu


def _random_problem(rng, nblocks, maxd):
    A = rng.standard_normal(2_000_000)
    B = rng.standard_normal(2_000_000)
    blocks, ref = [], []
    coff = 0
    aoff = boff = 0
    for _ in range(nblocks):
        m = int(rng.choice([1, 2, 7, 64, 65, 130, maxd]))
        n = int(rng.choice([1, 3, 63, 64, 129, maxd]))
        segs = []
        C = np.zeros((m, n))
        for _ in range(int(rng.integers(0, 4))):
            k = int(rng.choice([0, 1, 5, 16, 17, 100, maxd]))
            at, bt = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            lda = (m if at else k) + int(rng.integers(0, 3))
            ldb = (k if bt else n) + int(rng.integers(0, 3))
            lda, ldb = max(lda, 1), max(ldb, 1)
            alpha = float(rng.standard_normal())
            na = (k if at else m) * lda
            nb = (n if bt else k) * ldb
            Am = A[aoff:aoff + na].reshape(-1, lda)
            Bm = B[boff:boff + nb].reshape(-1, ldb)
            opA = Am[:k, :m].T if at else Am[:m, :k]
            opB = Bm[:n, :k].T if bt else Bm[:k, :n]
            C += alpha * opA @ opB
            segs.append((k, aoff, lda, at, boff, ldb, bt, alpha))
            aoff += na
            boff += nb
        blocks.append((m, n, coff, segs))
        ref.append((coff, C))
        coff += m * n
    return A, B, blocks, ref, coff


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grouped_gemm_fp64(seed):
    torch = cuda_torch()
    g = gpu_lib()
    rng = np.random.default_rng(seed)
    A, B, blocks, ref, ctot = _random_problem(rng, 12, 200)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((max(ctot, 1),), np.nan, dtype=torch.float64, device="cuda")
    g.grouped_gemm(g.DMRG_FP64, blocks, dA, dB, dC)
    C = dC.cpu().numpy()
    for (off, Cr), (m, n, _, _) in zip(ref, blocks):
        got = C[off:off + m * n].reshape(m, n)
        assert np.allclose(got, Cr, rtol=1e-13, atol=1e-12 * max(1.0, np.abs(Cr).max()))
