"""FP64-accurate products on the bf16 tensor cores (DMRG_FP64_TC): the grouped
GEMM against numpy FP64, the exactness of the integer slice sums in tensor
memory, per-row scaling over a wide dynamic range, and the FP64_TC sigma,
Davidson and sweep against the oracle.

Error model (per 64-deep stage, row scale 2^E_r of A, column scale 2^E_c of
B, six 8-bit slices): every element is represented to 2^(E-49); the dropped
slice products weigh 2^-48 of order 0 each.  So |C - AB| <= ~2^-45 sum over
stages of 64 2^(E_r + E_c), about 1e-13 K max|A_row| max|B_col|; the grouped
GEMM tests hold 1e-12 of that, sigma 1e-12 relative (the FP64 path's bar)."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle.dmrg import Oracle, davidson
from oracle.hamiltonian import eri_from_cholesky
from tests.helpers import cuda_torch, gpu_lib, make_case, rel_err

pytestmark = pytest.mark.gpu

FP64, BF16X3, FP64_TC = 0, 1, 4


def _blocks(rng, nblocks, A, B, kchoices=(1, 5, 63, 64, 65, 200, 700), int_range=None):
    """Ragged blocks with 0-3 segments (both orientations, padded leading
    dimensions, random alphas); returns the block list and exact products."""
    blocks, ref, bound = [], [], []
    coff = aoff = boff = 0
    for _ in range(nblocks):
        m = int(rng.choice([1, 7, 64, 127, 128, 129, 300]))
        n = int(rng.choice([1, 9, 63, 64, 65, 130]))
        nseg = int(rng.integers(0, 4))
        C = np.zeros((m, n))
        bnd = np.zeros((m, n))
        segs = []
        for _ in range(nseg):
            k = int(rng.choice(kchoices))
            at, bt = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            lda = (m if at else k) + int(rng.integers(0, 3))
            ldb = (k if bt else n) + int(rng.integers(0, 3))
            alpha = 1.0 if int_range else float(rng.standard_normal())
            na, nb = (k if at else m) * lda, (n if bt else k) * ldb
            Am = A[aoff:aoff + na].reshape(-1, lda)
            Bm = B[boff:boff + nb].reshape(-1, ldb)
            opA = Am[:k, :m].T if at else Am[:m, :k]
            opB = Bm[:n, :k].T if bt else Bm[:k, :n]
            if int_range:
                C += (opA.astype(np.int64) @ opB.astype(np.int64)).astype(np.float64)
            else:
                C += alpha * opA @ opB
            bnd += abs(alpha) * k * np.abs(opA).max(axis=1, initial=0)[:, None] * np.abs(opB).max(axis=0, initial=0)[None, :]
            segs.append((k, aoff, lda, at, boff, ldb, bt, alpha))
            aoff += na
            boff += nb
        blocks.append((m, n, coff, segs))
        ref.append((coff, m, n, C))
        bound.append(bnd)
        coff += m * n
    assert aoff <= A.size and boff <= B.size
    return blocks, ref, bound, coff


@pytest.mark.parametrize("seed", [1, 2])
def test_fp64_tc_grouped_gemm_vs_numpy(seed):
    torch = cuda_torch()
    g = gpu_lib()
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(4_000_000)
    B = rng.standard_normal(4_000_000)
    blocks, ref, bound, ctot = _blocks(rng, 24, A, B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((ctot,), np.nan, dtype=torch.float64, device="cuda")
    g.grouped_gemm(FP64_TC, blocks, dA, dB, dC)
    got = dC.cpu().numpy()
    worst = 0.0
    for (off, m, n, C), bnd in zip(ref, bound):
        G = got[off:off + m * n].reshape(m, n)
        assert np.all(np.isfinite(G))
        err = np.abs(G - C)
        assert np.all(err <= 1e-12 * bnd + 1e-300), float((err / np.maximum(bnd, 1e-300)).max())
        if bnd.max() > 0:
            worst = max(worst, float((err / np.maximum(bnd, 1e-300)).max()))
    print(f"seed {seed}: worst |err| / (K max|A_row| max|B_col|) = {worst:.2e}")


def test_fp64_tc_integer_products_are_exact():
    """Integer operands below 2^15: every stage's slice products are integers
    whose order sums stay below 2^24, so the result must equal the exact integer
    product bit for bit; a tensor-memory accumulation that rounded would not."""
    torch = cuda_torch()
    g = gpu_lib()
    rng = np.random.default_rng(7)
    A = rng.integers(-(1 << 15) + 1, 1 << 15, 2_000_000).astype(np.float64)
    B = rng.integers(-(1 << 15) + 1, 1 << 15, 2_000_000).astype(np.float64)
    blocks, ref, _, ctot = _blocks(rng, 16, A, B, kchoices=(1, 17, 64, 65, 300), int_range=True)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((ctot,), np.nan, dtype=torch.float64, device="cuda")
    g.grouped_gemm(FP64_TC, blocks, dA, dB, dC)
    got = dC.cpu().numpy()
    for off, m, n, C in ref:
        assert np.array_equal(got[off:off + m * n].reshape(m, n), C)


def test_fp64_tc_rows_and_columns_over_a_wide_range():
    """Rows of A scaled by 10^-8 .. 10^8 and columns of B by 10^-4 .. 10^4: the
    per-row / per-column scales keep every element's relative accuracy."""
    torch = cuda_torch()
    g = gpu_lib()
    rng = np.random.default_rng(3)
    m, k, n = 200, 500, 130
    A = rng.standard_normal((m, k)) * np.logspace(-8, 8, m)[:, None]
    B = rng.standard_normal((k, n)) * np.logspace(-4, 4, n)[None, :]
    C = A @ B
    dA = torch.from_numpy(A.ravel().copy()).cuda()
    dB = torch.from_numpy(B.ravel().copy()).cuda()
    dC = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    g.grouped_gemm(FP64_TC, [(m, n, 0, [(k, 0, k, 0, 0, n, 0, 1.0)])], dA, dB, dC)
    got = dC.cpu().numpy().reshape(m, n)
    scale = k * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    rel = np.abs(got - C) / scale
    print(f"wide range: worst error / (K max|A_row| max|B_col|) = {rel.max():.2e}")
    assert rel.max() <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_fp64_tc_sigma_small_every_bond(tmp_path, k):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D = 5, 5, 1, 10
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=FP64_TC)
    plan.set_bond(k)
    psi = si.random_vector(plan.dim, seed=1)
    x = torch.from_numpy(psi.copy()).cuda()
    y = torch.empty_like(x)
    plan.sigma(x, y)
    got = y.cpu().numpy()
    ref = ts.sigma(psi)
    print(f"K=5 bond {k}: FP64_TC sigma rel err {rel_err(got, ref):.2e}")
    assert rel_err(got, ref) <= 1e-12
    plan.close()


def test_fp64_tc_sigma_multi_tile(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 14, 14, 0, 600, 7
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split="gaussian", wn=1.0, ws=1.0)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=FP64_TC)
    plan.set_bond(k)
    psi = si.random_vector(plan.dim, seed=1)
    x = torch.from_numpy(psi.copy()).cuda()
    y = torch.empty_like(x)
    plan.sigma(x, y)
    got = y.cpu().numpy()
    ref = ts.sigma(psi)
    print(f"K=14 D=600: FP64_TC sigma rel err {rel_err(got, ref):.2e}")
    assert rel_err(got, ref) <= 1e-12
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    # the same stored operators on the FP64 arithmetic units
    z = torch.empty_like(x)
    plan.sigma_fp64_units(x, z)
    units = z.cpu().numpy()
    print(f"K=14 D=600: FP64 units sigma rel err {rel_err(units, ref):.2e}, vs FP64_TC {rel_err(got, units):.2e}")
    assert rel_err(units, ref) <= 1e-12
    plan.close()


def test_fp64_tc_davidson_and_full_D_sweep(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess[None], 1, 1e-9, 300)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=FP64_TC)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 1, tol=1e-8, max_iter=300)
    print(f"FP64_TC Davidson: dE = {e[0] - th_ref[0]:.2e} ({it} iterations)")
    assert conv and abs(e[0] - th_ref[0]) < 1e-9
    plan.close()
    # full-D sweeps reproduce FCI (the golden value written by the oracle)
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.txt")
    efci = [float(x) for line in open(gold) if line.startswith("k8_n8 ") for x in line.split(":")[1].split()][0]
    h, L, mps, path = make_case(tmp_path, K, N, twoS, 256, center=1)
    plan = g.Plan(h, L, K, N, twoS, 256, path, precision=FP64_TC, tol=1e-8)
    en, w = plan.sweep(2)
    print(f"FP64_TC full-D sweep K=8: E - E_FCI = {en[-1] - efci:.2e}")
    assert abs(en[-1] - efci) < 1e-9
    plan.close()


def test_refined_mixed_with_fp64_tc_store(tmp_path):
    """BF16X3 sigma over an FP64 store renormalised on the FP64 tensor-core
    engine, with the FP64 residual correction also on that engine: converged
    on the FP64-accurate residual, energy within 1e-6 Eh of the oracle."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess[None], 1, 1e-10, 300)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=BF16X3, fp64_store=1, fp64_tc=1, refine=1)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 1, tol=1e-7, max_iter=300)
    st = plan.stats()
    print(f"refined (FP64_TC store): dE = {e[0] - th_ref[0]:.2e}, {it} iterations, "
          f"{st['davidson_refine_last']} rounds, residual {st['davidson_rnorm_last']:.2e}")
    assert conv and abs(e[0] - th_ref[0]) < 1e-6
    plan.close()
