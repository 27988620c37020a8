"""dmrg_grouped_gemm_noalloc (work list in a static device array) against the
allocating FP64 entry point dmrg_grouped_gemm on the same products.

The file name sorts last so that the static-array variant also runs after
every other GPU test has used the device; it passes alone as well."""
import numpy as np
import pytest

from tests.helpers import cuda_torch, gpu_lib

pytestmark = pytest.mark.gpu


def _problem(seed, nblocks):
    """Ragged blocks (1..300), 0-3 segments each (an empty list gives a zero
    block), both operand orientations, padded leading dimensions."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(2_000_000)
    B = rng.standard_normal(2_000_000)
    blocks, ref = [], []
    coff = aoff = boff = 0
    for _ in range(nblocks):
        m = int(rng.choice([1, 7, 64, 65, 130, 300]))
        n = int(rng.choice([1, 9, 64, 100, 257]))
        nseg = int(rng.integers(0, 4))
        C = np.zeros((m, n))
        segs = []
        for _ in range(nseg):
            k = int(rng.choice([1, 5, 16, 63, 200]))
            at, bt = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            lda = (m if at else k) + int(rng.integers(0, 3))
            ldb = (k if bt else n) + int(rng.integers(0, 3))
            alpha = float(rng.standard_normal())
            na, nb = (k if at else m) * lda, (n if bt else k) * ldb
            Am = A[aoff:aoff + na].reshape(-1, lda)
            Bm = B[boff:boff + nb].reshape(-1, ldb)
            opA = Am[:k, :m].T if at else Am[:m, :k]
            opB = Bm[:n, :k].T if bt else Bm[:k, :n]
            C += alpha * opA @ opB
            segs.append((k, aoff, lda, at, boff, ldb, bt, alpha))
            aoff += na
            boff += nb
        blocks.append((m, n, coff, segs))
        ref.append((coff, m, n, C))
        coff += m * n
    assert aoff <= A.size and boff <= B.size
    return A, B, blocks, ref, coff


def test_noalloc_matches_allocating_entry_point():
    torch = cuda_torch()
    g = gpu_lib()
    probs = [_problem(11, 12), _problem(12, 9)]
    dev = []
    for A, B, blocks, ref, ctot in probs:
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        c_ref = torch.full((ctot,), np.nan, dtype=torch.float64, device="cuda")
        g.grouped_gemm(0, blocks, dA, dB, c_ref)  # allocating entry point (synchronises)
        c_new = torch.full((ctot,), np.nan, dtype=torch.float64, device="cuda")
        dev.append((dA, dB, blocks, ref, c_ref, c_new))
    # first call: set-up (symbol lookup; with lazy module loading the driver
    # also places the static array in device memory now)
    warm = torch.empty_like(dev[0][5])
    g.grouped_gemm_noalloc(dev[0][2], dev[0][0], dev[0][1], warm)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # two calls in a row on one stream, no synchronisation between them: the
    # second rewrites the static work list after the first kernel has read it
    for dA, dB, blocks, _, _, c_new in dev:
        g.grouped_gemm_noalloc(blocks, dA, dB, c_new)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across the allocation-free calls"
    assert torch.equal(warm, dev[0][5])
    for _, _, _, ref, c_ref, c_new in dev:
        got, exp = c_new.cpu().numpy(), c_ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        # same kernel and summation order as the allocating path
        np.testing.assert_allclose(got, exp, rtol=1e-14, atol=1e-14)
        for off, m, n, C in ref:
            np.testing.assert_allclose(got[off:off + m * n].reshape(m, n), C, rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_work_list_beyond_static_array():
    torch = cuda_torch()
    g = gpu_lib()
    limit = g.noalloc_scratch_bytes()
    assert limit == 4 << 20
    # a 1 x (64 * ntiles) block has ntiles 64-wide tiles of 48 bytes: just over
    # the limit.  The buffers are sized for the product, so nothing would be
    # out of bounds even if the check let it through.
    ntiles = limit // 48 + 64
    n = 64 * ntiles
    dA = torch.zeros(8, dtype=torch.float64, device="cuda")
    dB = torch.zeros(8 * n, dtype=torch.float64, device="cuda")
    dC = torch.zeros(n, dtype=torch.float64, device="cuda")
    blocks = [(1, n, 0, [(8, 0, 8, 0, 0, n, 0, 1.0)])]
    with pytest.raises(g.DMRGError) as exc:
        g.grouped_gemm_noalloc(blocks, dA, dB, dC)
    assert exc.value.code == -1 and "static scratch" in str(exc.value)


def test_noalloc_refuses_a_capturing_stream():
    """The work list is copied from host memory that the call frees on return,
    so a graph captured around the call would replay a dead host pointer.  A
    stream under capture is refused before anything is enqueued, and the
    entry point keeps working afterwards."""
    torch = cuda_torch()
    g = gpu_lib()
    A, B, blocks, ref, ctot = _problem(13, 4)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros(ctot, dtype=torch.float64, device="cuda")
    g.grouped_gemm_noalloc(blocks, dA, dB, dC)  # set-up outside any capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.stream(s):
        graph.capture_begin(capture_error_mode="thread_local")
        try:
            g.grouped_gemm_noalloc(blocks, dA, dB, dC, stream=s)
        except g.DMRGError as e:
            code = e.code
        finally:
            graph.capture_end()
    assert code == -1
    dC.zero_()
    g.grouped_gemm_noalloc(blocks, dA, dB, dC)
    got = dC.cpu().numpy()
    for off, m, n, C in ref:
        np.testing.assert_allclose(got[off:off + m * n].reshape(m, n), C, rtol=1e-12, atol=1e-12)
