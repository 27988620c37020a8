"""Learned Davidson preconditioner on the GPU: forward and gradient kernels
against the oracle's FP64 network, training on harvested Jacobi-Davidson pairs,
and Davidson with the trained network against the plain (Jacobi) method."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import mlp as omlp
from oracle.dmrg import Oracle, davidson
from oracle.hamiltonian import eri_from_cholesky
from tests.helpers import cuda_torch, gpu_lib, make_case

pytestmark = pytest.mark.gpu


def _plan(tmp_path, K=8, N=8, D=64, k=4, precision=0):
    g = gpu_lib()
    h, L, mps, path = make_case(tmp_path, K, N, 0, D, center=k)
    plan = g.Plan(h, L, K, N, 0, D, path, precision=precision)
    plan.set_bond(k)
    return plan, h, L, mps


def test_forward_and_gradient_match_oracle(tmp_path):
    torch = cuda_torch()
    plan, *_ = _plan(tmp_path)
    rng = np.random.default_rng(5)
    theta = (rng.standard_normal(omlp.N_PARAMS) * 0.3).astype(np.float32)
    plan.mlp_params(theta)
    assert np.array_equal(plan.mlp_params(), theta)
    X = rng.standard_normal((1000, 5)).astype(np.float32)
    y = rng.standard_normal(1000).astype(np.float32)
    g_ref, _, _ = omlp.forward(theta.astype(np.float64), X.astype(np.float64))
    L_ref, grad_ref = omlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    dX, dy = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    dg = torch.empty(1000, dtype=torch.float32, device="cuda")
    plan.mlp_eval(dX, dg)
    got = dg.cpu().numpy()
    assert np.max(np.abs(got - g_ref)) <= 1e-5 * (1 + np.max(np.abs(g_ref)))
    plan.mlp_eval(dX, dg, bf16=True)  # bf16 weights: within the bf16 rounding of the parameters
    assert np.max(np.abs(dg.cpu().numpy() - g_ref)) <= 3e-2 * (1 + np.max(np.abs(g_ref)))
    dgrad = torch.empty(omlp.N_PARAMS, dtype=torch.float32, device="cuda")
    dloss = torch.empty(1, dtype=torch.float32, device="cuda")
    plan.mlp_gradient(dX, dy, dgrad, dloss)
    grad = dgrad.cpu().numpy()
    assert abs(float(dloss.item()) - L_ref) <= 1e-5 * L_ref
    assert np.max(np.abs(grad - grad_ref)) <= 1e-4 * (1e-3 + np.max(np.abs(grad_ref)))
    plan.close()


def test_training_on_harvested_pairs_reduces_the_loss(tmp_path):
    torch = cuda_torch()
    plan, *_ = _plan(tmp_path)
    plan.mlp_init(3)
    x = torch.from_numpy(si.random_vector(plan.dim, seed=1)).cuda()
    e, n_pairs = plan.mlp_harvest(x, max_iter=12, jd_iters=60, per_solve=4096)
    print(f"harvest: E = {e:.10f}, {n_pairs} pairs")
    assert n_pairs > 1000
    l0, l1 = plan.mlp_train(steps=300, batch=2048, lr=3e-3, seed=11)
    print(f"training loss {l0:.4e} -> {l1:.4e}")
    # the per-element targets are noisy functions of the five inputs: the network
    # can only learn their conditional mean, so the loss falls but not to zero
    assert np.isfinite(l1) and l1 < l0
    plan.close()


def test_trained_preconditioner_against_jacobi(tmp_path):
    """Same bond, same guess: Davidson with the trained g against plain Jacobi.
    Both reach the oracle eigenvalue; the iteration counts are reported."""
    torch = cuda_torch()
    K, N, D, k = 10, 10, 128, 5
    plan, h, L, mps = _plan(tmp_path, K=K, N=N, D=D, k=k)
    ts = Oracle(h, eri_from_cholesky(L), N, 0, mps).two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess[None], 1, 1e-10, 400)
    plan.mlp_init(3)
    for seed in (21, 22, 23):  # pairs from plain runs started at other guesses
        x = torch.from_numpy(si.random_vector(ts.dim, seed=seed)).cuda()
        plan.mlp_harvest(x, max_iter=15, jd_iters=60, per_solve=8192)
    l0, l1 = plan.mlp_train(steps=600, batch=4096, lr=3e-3, seed=7)
    res = {}
    for name, pc in (("jacobi", 0), ("mlp", 1)):
        x = torch.from_numpy(guess.copy()).cuda()
        e, it, conv = plan.davidson(x, 1, tol=1e-6, max_iter=300, precond=pc)
        res[name] = (e[0], it)
        assert abs(e[0] - th_ref[0]) < 1e-8
    st = plan.stats()
    print(f"loss {l0:.3e} -> {l1:.3e}; Davidson iterations to |r| <= 1e-6: jacobi {res['jacobi'][1]}, "
          f"mlp {res['mlp'][1]}; fallbacks {st['precond_fallbacks']}")
    plan.close()
