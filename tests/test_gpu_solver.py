"""GPU parity of Davidson (FP64 on the device), decimation and sweeps.

Energies are gauge invariant; decimation is compared through its discarded
weight and the lowest H_eff eigenvalue at the next bond, both from the same
seeded two-site vector (input generator, seed 11)."""
import os

import numpy as np
import pytest

import synthetic_inputs as si
from oracle.dmrg import Oracle, davidson
from oracle.hamiltonian import eri_from_cholesky
from tests.helpers import cuda_torch, gpu_lib, make_case

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.txt")


def golden(name):
    for line in open(GOLDEN):
        if line.startswith(name + " "):
            return [float(x) for x in line.split(":")[1].split()]
    raise KeyError(name)


def test_davidson_matches_oracle_eigenvalue(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    o = Oracle(h, eri_from_cholesky(L), N, twoS, mps)
    ts = o.two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess[None], 1, 1e-9, 300)
    plan = g.Plan(h, L, K, N, twoS, D, path)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 1, tol=1e-9, max_iter=300)
    assert conv
    assert abs(e[0] - th_ref[0]) < 1e-9
    # returned vector is a normalised eigenvector
    y = torch.empty_like(x)
    plan.sigma(x, y)
    xv, yv = x.cpu().numpy(), y.cpu().numpy()
    assert abs(np.linalg.norm(xv) - 1) < 1e-10
    assert np.linalg.norm(yv - e[0] * xv) < 1e-8
    plan.close()


def test_davidson_two_roots(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 6, 6, 0, 64, 3
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    o = Oracle(h, eri_from_cholesky(L), N, twoS, mps)
    ts = o.two_site(k)
    guess = si.random_vector(ts.dim, seed=1, nvec=2)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess, 2, 1e-9, 300)
    plan = g.Plan(h, L, K, N, twoS, D, path)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 2, tol=1e-9, max_iter=300)
    assert conv
    assert np.allclose(e, th_ref, atol=1e-9)
    plan.close()


@pytest.mark.parametrize("forward", [True, False])
def test_decimation_and_next_bond(tmp_path, forward):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    Dcut = 20
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    o = Oracle(h, eri_from_cholesky(L), N, twoS, mps)
    ts = o.two_site(k)
    psi = si.random_vector(ts.dim, seed=11)
    w_ref, guess_ref = o.decimate_and_move(ts, k, psi[None], Dcut, forward)
    kn = k + 1 if forward else k - 1
    ts2 = o.two_site(kn)
    g_ref = guess_ref[0]
    rq_ref = g_ref @ ts2.sigma(g_ref) / (g_ref @ g_ref)
    th_ref, _, _ = davidson(ts2.sigma, ts2.hdiag(), guess_ref, 1, 1e-9, 300)

    plan = g.Plan(h, L, K, N, twoS, D, path)
    plan.set_bond(k)
    x = torch.from_numpy(psi.copy()).cuda()
    cap = 4 * ts.dim
    nxt = torch.zeros(cap, dtype=torch.float64, device="cuda")
    w, ndim = plan.decimate(x, 1, Dcut, forward, next_psi=nxt, next_cap=cap)
    assert abs(w - w_ref) < 1e-12
    assert ndim == ts2.dim and plan.dim == ts2.dim
    gv = nxt[:ndim].clone()
    sg = torch.empty_like(gv)
    plan.sigma(gv, sg)
    gn = float(gv @ gv)
    assert abs(gn - g_ref @ g_ref) < 1e-10
    assert abs(float(gv @ sg) / gn - rq_ref) < 1e-10
    e, it, conv = plan.davidson(gv, 1, tol=1e-9, max_iter=300)
    assert conv
    assert abs(e[0] - th_ref[0]) < 1e-9
    plan.close()


def test_full_D_sweep_matches_fci(tmp_path):
    cuda_torch()
    g = gpu_lib()
    K, N, twoS, D = 6, 6, 0, 64
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=1)
    plan = g.Plan(h, L, K, N, twoS, D, path, tol=1e-8)
    e, w = plan.sweep(2)
    assert abs(e[-1] - golden("k6_n6")[0]) < 1e-10
    plan.close()


def test_k8_sweeps_vs_fci(tmp_path):
    """K=8, N=8 (4900 determinants): D=64 stays variational, D=256 reaches FCI."""
    cuda_torch()
    g = gpu_lib()
    K, N, twoS = 8, 8, 0
    efci = golden("k8_n8")[0]
    h, L, mps, path = make_case(tmp_path, K, N, twoS, 64, center=1)
    plan = g.Plan(h, L, K, N, twoS, 64, path, tol=1e-7)
    e, w = plan.sweep(4)
    assert e[-1] >= efci - 1e-10
    assert e[-1] - efci < 5e-3
    plan.close()
    h, L, mps, path = make_case(tmp_path, K, N, twoS, 256, center=1)
    plan = g.Plan(h, L, K, N, twoS, 256, path, tol=1e-8)
    e, w = plan.sweep(2)
    assert abs(e[-1] - efci) < 1e-10
    plan.close()


@pytest.mark.parametrize("forward", [True, False])
def test_decimation_two_stage_eigensolver(tmp_path, forward):
    """Density-matrix blocks of 256 rows or more take the two-stage eigensolver
    (FP32 sweeps, FP64 basis change and FP64 sweeps): discarded weight and the
    next-bond guess against the oracle's dense FP64 decomposition."""
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 14, 14, 0, 600, 7
    Dcut = 300
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split="gaussian", wn=1.0, ws=1.0)
    o = Oracle(h, eri_from_cholesky(L), N, twoS, mps)
    ts = o.two_site(k)
    psi = si.random_vector(ts.dim, seed=11)
    w_ref, guess_ref = o.decimate_and_move(ts, k, psi[None], Dcut, forward)
    g_ref = guess_ref[0]

    plan = g.Plan(h, L, K, N, twoS, D, path)
    plan.set_bond(k)
    x = torch.from_numpy(psi.copy()).cuda()
    cap = 4 * ts.dim
    nxt = torch.zeros(cap, dtype=torch.float64, device="cuda")
    w, ndim = plan.decimate(x, 1, Dcut, forward, next_psi=nxt, next_cap=cap)
    st = plan.stats()
    print(f"K=14 D=600 -> {Dcut}: blocks {st['decim_nmat_last']}, largest {st['decim_nmax_last']}, "
          f"sweeps FP32 {st['decim_sweeps32_last']} + FP64 {st['decim_sweeps_last']}, w {w:.15e} vs {w_ref:.15e}")
    assert st["decim_nmax_last"] >= 256 and st["decim_sweeps32_last"] > 0
    assert abs(w - w_ref) < 1e-12 * max(1.0, abs(w_ref))
    gv = nxt[:ndim].cpu().numpy()
    assert ndim == g_ref.size
    # the guess is defined up to the gauge of the kept basis: compare its norm
    # and its energy at the next bond
    assert abs(gv @ gv - g_ref @ g_ref) < 1e-10
    ts2 = o.two_site(k + 1 if forward else k - 1)
    rq_ref = g_ref @ ts2.sigma(g_ref) / (g_ref @ g_ref)
    gt = torch.from_numpy(gv.copy()).cuda()
    sg = torch.empty_like(gt)
    plan.sigma(gt, sg)
    assert abs(float(gt @ sg) / float(gt @ gt) - rq_ref) < 1e-9
    plan.close()
