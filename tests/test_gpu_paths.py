"""GPU parity of configurations the full-size workload runs and the smaller
parity cases do not reach by default, against the CPU oracle.

* sigma lowered into several scratch chunks (the K=73 middle bond needs ten;
  the automatic scratch floor keeps every small case in one), FP64 engine and
  tensor cores;
* tensor-core sigma of several vectors per launch (Davidson blocks, roots);
* sectors wider than 256 (the K=73, D=3000 middle bond reaches ~440);
* two-root mixed-precision Davidson with the FP64 residual correction and the
  state-averaged decimation of its vectors;
* the FP64 residual correction itself (Davidson converged on the FP64
  residual, energies within 1e-6 Eh of the oracle)."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle.dmrg import Oracle, davidson
from oracle.hamiltonian import eri_from_cholesky
from tests.helpers import cuda_torch, gpu_lib, make_case, rel_err

pytestmark = pytest.mark.gpu

FP64, BF16X3 = 0, 1
# mixed-mode bound measured for BF16X3 with the tensor-core operator store at
# K=14 (1.1e-5; above the 1e-5 target, which fp64_store meets)
TOL_MIXED = 2e-5


def _oracle_sigma(h, L, N, twoS, mps, k, nvec=1, seed=1):
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    psi = si.random_vector(ts.dim, seed=seed, nvec=nvec).reshape(nvec, ts.dim)
    return ts, psi, np.array([ts.sigma(p) for p in psi])


@pytest.mark.parametrize("prec", [FP64, BF16X3])
def test_sigma_in_several_scratch_chunks(tmp_path, prec):
    """K=14, D=600 middle bond with a 4 MB scratch: the product list is lowered
    into >= 3 chunks (phase-1 products of each chunk in scratch, then its
    fused term sums), as at the K=73 middle bond."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 14, 14, 0, 600, 7
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split="gaussian", wn=1.0, ws=1.0)
    ts, psi, ref = _oracle_sigma(h, L, N, twoS, mps, k)
    out = {}
    for sb in (0, 4 << 20):
        plan = g.Plan(h, L, K, N, twoS, D, path, precision=prec, scratch_bytes=sb)
        plan.set_bond(k)
        chunks = plan.stats()["sigma_chunks"]
        x = torch.from_numpy(psi[0].copy()).cuda()
        y = torch.empty_like(x)
        plan.sigma(x, y)
        torch.cuda.synchronize()
        out[sb] = (chunks, y.cpu().numpy())
        plan.close()
    assert out[0][0] == 1 and out[4 << 20][0] >= 3, (out[0][0], out[4 << 20][0])
    got = out[4 << 20][1]
    bound = 1e-12 if prec == FP64 else TOL_MIXED
    print(f"prec={prec}: {out[4 << 20][0]} chunks, rel err {rel_err(got, ref[0]):.2e}")
    assert rel_err(got, ref[0]) <= bound
    assert np.abs(got - ref[0]).max() <= (1e-11 if prec == FP64 else 1e-3) * np.abs(ref[0]).max()
    # chunking reorders FP64 additions only
    assert rel_err(got, out[0][1]) <= (1e-14 if prec == FP64 else 1e-5)


def test_sigma_one_launch_pair_per_term(tmp_path):
    """sigma_per_term = 1 (the launch-per-term baseline): one scratch chunk per
    Hamiltonian term, so as many launch pairs as terms with products; the
    result equals the oracle's like the grouped launch's."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    ts, psi, ref = _oracle_sigma(h, L, N, twoS, mps, k)
    res = {}
    for pt in (0, 1):
        plan = g.Plan(h, L, K, N, twoS, D, path, precision=1, sigma_per_term=pt, sigma_tile_n=128)
        plan.set_bond(k)
        st = plan.stats()
        x = torch.from_numpy(psi[0].copy()).cuda()
        y = torch.empty_like(x)
        plan.sigma(x, y)
        torch.cuda.synchronize()
        res[pt] = (st["sigma_chunks"], st["n_terms"], y.cpu().numpy())
        plan.close()
    print(f"launch pairs: grouped {res[0][0]}, per term {res[1][0]} ({res[1][1]} terms); "
          f"rel err {rel_err(res[1][2], ref[0]):.2e}")
    assert res[0][0] == 1 and res[1][0] > 10 * res[0][0] and res[1][0] <= res[1][1]
    assert rel_err(res[1][2], ref[0]) <= TOL_MIXED


def test_tensor_core_sigma_three_vectors_per_launch(tmp_path):
    """n_roots = 3: the mixed sigma launches three vectors per grouped launch;
    each is compared element by element with the oracle and with one-vector
    calls of the same plan."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 14, 14, 0, 600, 7
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split="gaussian", wn=1.0, ws=1.0)
    ts, psi, ref = _oracle_sigma(h, L, N, twoS, mps, k, nvec=3)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=BF16X3, n_roots=3)
    plan.set_bond(k)
    dim = plan.dim
    x = torch.from_numpy(psi.copy()).cuda()
    y = torch.empty_like(x)
    plan.sigma(x, y, nvec=3)
    y1 = torch.empty_like(x)
    for v in range(3):
        plan.sigma(x[v], y1[v])
    torch.cuda.synchronize()
    got, one = y.cpu().numpy(), y1.cpu().numpy()
    for v in range(3):
        e = rel_err(got[v], ref[v])
        print(f"vector {v}: rel err {e:.2e}")
        assert e <= TOL_MIXED
        assert np.abs(got[v] - ref[v]).max() <= 1e-3 * np.abs(ref[v]).max()
        # same tiles and products; only the order of the FP64 drains may differ
        assert rel_err(got[v], one[v]) <= 1e-12
    assert dim == ts.dim
    plan.close()


def test_sigma_sectors_wider_than_256(tmp_path):
    """K=14, D=1000, Gaussian split of width 0.6: left and right sectors of 400
    states (each output block spans four 128-row tiles), FP64 and tensor cores."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 14, 14, 0, 1000, 7
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split="gaussian", wn=0.6, ws=0.6)
    ts, psi, ref = _oracle_sigma(h, L, N, twoS, mps, k)
    assert max(s[5] for s in ts.layout) > 256 and max(s[6] for s in ts.layout) > 256
    for prec, bound in [(FP64, 1e-12), (BF16X3, TOL_MIXED)]:
        plan = g.Plan(h, L, K, N, twoS, D, path, precision=prec)
        plan.set_bond(k)
        x = torch.from_numpy(psi[0].copy()).cuda()
        y = torch.empty_like(x)
        plan.sigma(x, y)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        print(f"K=14 D=1000 prec={prec}: rel err {rel_err(got, ref[0]):.2e}")
        assert rel_err(got, ref[0]) <= bound
        plan.close()


def test_refined_mixed_davidson_k8(tmp_path):
    """BF16X3 sigma over the FP64 store with the FP64 residual correction:
    Davidson converges on the FP64 residual (tol 1e-7) and the energy is
    within 1e-6 Eh of the oracle's FP64 Davidson; the same BF16X3 Davidson
    without the correction stops at its noise floor."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess[None], 1, 1e-10, 300)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=BF16X3, fp64_store=1, refine=1)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 1, tol=1e-7, max_iter=300)
    st = plan.stats()
    print(f"refined: dE = {e[0] - th_ref[0]:.2e}, {it} mixed iterations, {st['davidson_refine_last']} rounds, "
          f"FP64 residual {st['davidson_rnorm_last']:.2e}, {st['sigma_acc_calls']} FP64 sigma")
    assert conv and st["davidson_conv_last"] == 1
    assert st["davidson_rnorm_last"] <= 1e-7
    assert st["davidson_refine_last"] >= 1
    assert abs(e[0] - th_ref[0]) < 1e-6
    # the returned vector's FP64 residual, formed here from the FP64 sigma
    z = torch.empty_like(x)
    plan.sigma_fp64(x, z)
    xv, zv = x.cpu().numpy(), z.cpu().numpy()
    assert np.linalg.norm(zv - e[0] * xv) <= 2e-7
    plan.close()
    plain = g.Plan(h, L, K, N, twoS, D, path, precision=BF16X3, fp64_store=1)
    plain.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e2, it2, conv2 = plain.davidson(x, 1, tol=1e-7, max_iter=300)
    st2 = plain.stats()
    print(f"plain mixed: dE = {e2[0] - th_ref[0]:.2e}, {it2} iterations, stalled {st2['davidson_stalled_last']}, "
          f"residual {st2['davidson_rnorm_last']:.2e}")
    assert not conv2 and st2["davidson_stalled_last"] == 1 and it2 < 300
    plain.close()


def test_refined_mixed_davidson_k14(tmp_path):
    """The same at K=14, D=600 (multi-tile blocks): the FP64 residual meets
    1e-6, and the energy is the oracle's Rayleigh quotient of the returned
    vector, whose oracle residual is also <= 1.5e-6."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 14, 14, 0, 600, 7
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split="gaussian", wn=1.0, ws=1.0)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=BF16X3, fp64_store=1, refine=1)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 1, tol=1e-6, max_iter=300)
    st = plan.stats()
    assert conv and st["davidson_rnorm_last"] <= 1e-6
    # the oracle's Rayleigh quotient and residual of the returned vector
    xv = x.cpu().numpy()
    sv = ts.sigma(xv)
    rq = xv @ sv / (xv @ xv)
    print(f"K=14 refined: E {e[0]:.10f}, oracle RQ {rq:.10f}, dE {e[0] - rq:.2e}, "
          f"oracle residual {np.linalg.norm(sv - rq * xv):.2e}, {it} iterations, "
          f"{st['davidson_refine_last']} rounds")
    # E is the oracle's Rayleigh quotient of the vector, and the oracle's
    # residual bounds its distance to the eigenvalue by |r|^2 / gap
    assert abs(e[0] - rq) < 1e-8
    assert np.linalg.norm(sv - rq * xv) <= 1.5e-6
    plan.close()


def test_refined_two_roots_and_state_averaged_decimation(tmp_path):
    """Two roots: mixed Davidson with the FP64 residual correction against the
    oracle's two eigenvalues, then the state-averaged decimation of those two
    vectors against the oracle's decimation of the same vectors."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k, Dcut = 8, 8, 0, 64, 4, 20
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    o = Oracle(h, eri_from_cholesky(L), N, twoS, mps)
    ts = o.two_site(k)
    guess = si.random_vector(ts.dim, seed=1, nvec=2).reshape(2, ts.dim)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess, 2, 1e-10, 300)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=BF16X3, fp64_store=1, refine=1, n_roots=2)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 2, tol=1e-7, max_iter=300)
    print(f"two roots refined: dE = {e - th_ref[:2]}, {it} iterations")
    assert conv
    assert np.allclose(e, th_ref[:2], atol=1e-6)
    X = x.cpu().numpy().reshape(2, -1)
    w_ref, guess_ref = o.decimate_and_move(ts, k, X, Dcut, True)
    cap = 8 * ts.dim
    nxt = torch.zeros(cap, dtype=torch.float64, device="cuda")
    w, ndim = plan.decimate(x, 2, Dcut, True, next_psi=nxt, next_cap=cap // 2)
    print(f"state-averaged discarded weight {w:.6e} (oracle {w_ref:.6e})")
    assert abs(w - w_ref) < 1e-12
    ts2 = o.two_site(k + 1)
    assert ndim == ts2.dim
    # gauge-invariant check of the next-bond guesses (each side in its own
    # basis of the new bond): their Gram matrix and their 2 x 2 H_eff matrix,
    # the library's from its FP64-arithmetic sigma over its FP64 store
    gdev = nxt[:2 * ndim].reshape(2, ndim).contiguous()
    hdev = torch.empty_like(gdev)
    plan.sigma_fp64(gdev, hdev, nvec=2)
    gv, hg = gdev.cpu().numpy(), hdev.cpu().numpy()
    gr = guess_ref
    hr = np.array([ts2.sigma(v) for v in gr])
    np.testing.assert_allclose(gv @ gv.T, gr @ gr.T, atol=1e-10)
    np.testing.assert_allclose(gv @ hg.T, gr @ hr.T, atol=1e-9)
    plan.close()


def test_bond_update_from_host_buffers_matches_device_calls(tmp_path):
    """dmrg_update_bond_host (guess in and next guess out through host memory)
    against dmrg_davidson + dmrg_decimate on device buffers, from the same guess:
    same energy, discarded weight and next-bond guess (FP64)."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k, Dcut = 8, 8, 0, 64, 4, 20
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    guess = si.random_vector(make_dim(g, h, L, K, N, twoS, D, path, k), seed=3)
    res = []
    for host in (False, True):
        plan = g.Plan(h, L, K, N, twoS, D, path, tol=1e-9, max_iter=300)
        plan.set_bond(k)
        cap = 4 * plan.dim
        if host:
            nxt = np.zeros(cap)
            e, it, w, nd, conv = plan.update_bond_host(guess.copy(), 1, Dcut, True, next_psi=nxt)
            res.append((e[0], w, nxt[:nd].copy()))
        else:
            x = torch.from_numpy(guess.copy()).cuda()
            e, it, conv = plan.davidson(x, 1, tol=1e-9, max_iter=300)
            dn = torch.zeros(cap, dtype=torch.float64, device="cuda")
            w, nd = plan.decimate(x, 1, Dcut, True, next_psi=dn, next_cap=cap)
            res.append((e[0], w, dn[:nd].cpu().numpy()))
        assert conv
        plan.close()
    (e0, w0, g0), (e1, w1, g1) = res
    assert abs(e0 - e1) < 1e-10 and abs(w0 - w1) < 1e-14
    assert g0.shape == g1.shape and np.allclose(g0, g1, rtol=0, atol=1e-10)


def make_dim(g, h, L, K, N, twoS, D, path, k):
    plan = g.Plan(h, L, K, N, twoS, D, path)
    plan.set_bond(k)
    d = plan.dim
    plan.close()
    return d


def test_plan_from_full_eri_array(tmp_path):
    """n_chol = 0: the plan takes the full (pq|rs) array; sigma equals the
    Cholesky-built plan's to rounding, and an array without the real-orbital
    symmetry is refused."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, k = 8, 8, 4
    h, L, mps, path = make_case(tmp_path, K, N, 0, 64, center=k)
    eri = eri_from_cholesky(L)
    ys = []
    for ints in (L, eri):
        plan = g.Plan(h, ints, K, N, 0, 64, path)
        plan.set_bond(k)
        x = torch.from_numpy(si.random_vector(plan.dim, seed=1)).cuda()
        y = torch.empty_like(x)
        plan.sigma(x, y)
        ys.append(y.cpu().numpy())
        plan.close()
    err = np.linalg.norm(ys[1] - ys[0]) / np.linalg.norm(ys[0])
    print(f"full (pq|rs) vs Cholesky plan: sigma rel diff {err:.2e}")
    assert err < 1e-13
    bad = eri.copy()
    bad[0, 1, 2, 3] += 1e-3
    with pytest.raises(g.DMRGError) as exc:
        g.Plan(h, bad, K, N, 0, 64, path)
    assert exc.value.code == -1
