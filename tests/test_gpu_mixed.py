"""Mixed-precision path (tcgen05 on bf16 pieces) against the FP64 oracle.

Which modes meet the mixed-path targets (sigma relative error <= 1e-5,
energies within 1e-6 Eh), as these tests measure them:
* BF16X3 sigma over an FP64 operator store (fp64_store = 1) meets the sigma
  target; with the FP64 Rayleigh quotient (fp64_final = 1) or the FP64
  residual correction (refine = 1, tests/test_gpu_paths.py) it meets the
  energy target.
* BF16X3 and BF16X6 with the operator store built on the tensor cores do NOT
  meet them: the FP32 accumulation in tensor memory (about 2^-23 per 16-deep
  MMA step, inherited by every later bond) leaves the store at a few 1e-6
  relative, and sigma at 1.1e-5 (K=14, BF16X3).  These tests hold those modes
  to their measured values -- sigma <= 1e-5 (small) and 2e-5 (multi-tile),
  energies <= 1e-4 Eh (BF16X3) and 5e-5 Eh (BF16X6) -- so that a regression
  shows; they are not a claim that the targets are met.
Plain BF16 is held to relative error <= 3e-2."""
import os

import numpy as np
import pytest

import synthetic_inputs as si
from oracle.dmrg import Oracle, davidson
from oracle.hamiltonian import eri_from_cholesky
from tests.helpers import cuda_torch, gpu_lib, make_case, rel_err

pytestmark = pytest.mark.gpu

BF16X3, BF16, BF16X6 = 1, 2, 3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.txt")


def _golden(name):
    for line in open(GOLDEN):
        if line.startswith(name + " "):
            return [float(x) for x in line.split(":")[1].split()]
    raise KeyError(name)


def _sigma_pair(tmp_path, precision, K, N, twoS, D, k, split="proportional", wn=None, ws=None, fp64_store=0):
    torch = cuda_torch()
    g = gpu_lib()
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split=split, wn=wn, ws=ws)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=precision, fp64_store=fp64_store)
    plan.set_bond(k)
    dim = plan.dim
    assert dim == ts.dim
    psi = si.random_vector(dim, seed=1)
    x = torch.from_numpy(psi.copy()).cuda()
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    plan.sigma(x, y)
    plan.sigma_fp64(x, z)
    torch.cuda.synchronize()
    ref = ts.sigma(psi)
    got, got64 = y.cpu().numpy(), z.cpu().numpy()
    plan.close()
    return rel_err(got, ref), rel_err(got, got64), rel_err(got64, ref)


@pytest.mark.parametrize("prec,bound", [(BF16X3, 1e-5), (BF16X6, 1e-5)])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_mixed_sigma_small(tmp_path, k, prec, bound):
    e_ref, e_arith, e_store = _sigma_pair(tmp_path, prec, 5, 5, 1, 10, k)
    print(f"K=5 k={k} prec={prec}: mixed vs oracle {e_ref:.2e}, vs fp64-arith {e_arith:.2e}, store {e_store:.2e}")
    assert e_ref <= bound


@pytest.mark.parametrize("prec,bound", [(BF16X3, 2e-5), (BF16X6, 1e-5)])
def test_mixed_sigma_multi_tile(tmp_path, prec, bound):
    e_ref, e_arith, e_store = _sigma_pair(tmp_path, prec, 14, 14, 0, 600, 7, "gaussian", 1.0, 1.0)
    print(f"K=14 D=600 prec={prec}: mixed vs oracle {e_ref:.2e}, vs fp64-arith {e_arith:.2e}, store {e_store:.2e}")
    assert e_ref <= bound


def test_bf16_sigma_multi_tile(tmp_path):
    e_ref, e_arith, e_store = _sigma_pair(tmp_path, BF16, 14, 14, 0, 600, 7, "gaussian", 1.0, 1.0)
    print(f"K=14 D=600 bf16: vs oracle {e_ref:.2e}, vs fp64-arith {e_arith:.2e}, store {e_store:.2e}")
    assert e_ref <= 3e-2


@pytest.mark.parametrize("prec,tols", [(BF16X3, (5e-4, 1e-4)), (BF16X6, (5e-4, 5e-5))])
def test_mixed_davidson_energy(tmp_path, prec, tols):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess[None], 1, 1e-9, 300)
    for fp64_final, tol in [(0, tols[0]), (1, tols[1])]:
        plan = g.Plan(h, L, K, N, twoS, D, path, precision=prec, fp64_final=fp64_final)
        plan.set_bond(k)
        x = torch.from_numpy(guess.copy()).cuda()
        e, it, conv = plan.davidson(x, 1, tol=1e-5, max_iter=300)
        print(f"mixed davidson prec={prec} fp64_final={fp64_final}: dE = {e[0] - th_ref[0]:.2e} ({it} iterations)")
        assert abs(e[0] - th_ref[0]) < tol
        plan.close()


@pytest.mark.parametrize("prec,tol", [(BF16X3, 1e-4), (BF16X6, 5e-5)])
def test_mixed_sweep_k8_full_D(tmp_path, prec, tol):
    cuda_torch()
    g = gpu_lib()
    K, N, twoS = 8, 8, 0
    efci = _golden("k8_n8")[0]
    h, L, mps, path = make_case(tmp_path, K, N, twoS, 256, center=1)
    plan = g.Plan(h, L, K, N, twoS, 256, path, precision=prec, tol=1e-5, fp64_final=1)
    e, w = plan.sweep(2)
    print(f"mixed full-D sweep K=8 prec={prec}: E - E_FCI = {e[-1] - efci:.2e}")
    assert abs(e[-1] - efci) < tol
    plan.close()


# FP64 operator store (renormalisation and intermediates on the FP64 engine)
# with bf16 piece copies for the tensor-core sigma: the mixed-mode targets.
def test_fp64_store_sigma_multi_tile(tmp_path):
    e_ref, e_arith, e_store = _sigma_pair(tmp_path, BF16X3, 14, 14, 0, 600, 7, "gaussian", 1.0, 1.0, fp64_store=1)
    print(f"K=14 D=600 BF16X3 + FP64 store: vs oracle {e_ref:.2e}, vs fp64-arith {e_arith:.2e}, store {e_store:.2e}")
    assert e_store <= 1e-12
    assert e_ref <= 1e-5


def test_fp64_store_davidson_energy(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    ts = Oracle(h, eri_from_cholesky(L), N, twoS, mps).two_site(k)
    guess = si.random_vector(ts.dim, seed=1)
    th_ref, _, _ = davidson(ts.sigma, ts.hdiag(), guess[None], 1, 1e-9, 300)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=BF16X3, fp64_store=1, fp64_final=1)
    plan.set_bond(k)
    x = torch.from_numpy(guess.copy()).cuda()
    e, it, conv = plan.davidson(x, 1, tol=1e-5, max_iter=300)
    print(f"BF16X3 + FP64 store davidson: dE = {e[0] - th_ref[0]:.2e} ({it} iterations)")
    assert abs(e[0] - th_ref[0]) < 1e-6
    plan.close()


def test_fp64_store_sweep_k8_full_D(tmp_path):
    cuda_torch()
    g = gpu_lib()
    K, N, twoS = 8, 8, 0
    efci = _golden("k8_n8")[0]
    h, L, mps, path = make_case(tmp_path, K, N, twoS, 256, center=1)
    plan = g.Plan(h, L, K, N, twoS, 256, path, precision=BF16X3, tol=1e-5, fp64_final=1, fp64_store=1)
    e, w = plan.sweep(2)
    print(f"BF16X3 + FP64 store full-D sweep K=8: E - E_FCI = {e[-1] - efci:.2e}")
    assert abs(e[-1] - efci) < 1e-6
    plan.close()
