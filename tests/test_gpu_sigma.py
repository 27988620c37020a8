"""GPU parity of the sigma product (Eq. Sigma) and diag(H_eff) with the CPU oracle.

The environments are built by the library's own renormalisation (Eq. Renorm)
from the same seeded MPS the oracle reads, so these cases also check the
renormalised operator store.  FP64 bar: relative 2-norm error <= 1e-12 and
element-wise |d| <= 1e-11 * max|sigma_ref|."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle.dmrg import Oracle
from oracle.hamiltonian import eri_from_cholesky
from tests.helpers import cuda_torch, gpu_lib, make_case, rel_err

pytestmark = pytest.mark.gpu

TOL_REL = 1e-12
TOL_ELT = 1e-11


def _compare_bond(tmp_path, K, N, twoS, D, k, split="proportional", wn=None, ws=None, nvec=1):
    torch = cuda_torch()
    g = gpu_lib()
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k, split=split, wn=wn, ws=ws)
    o = Oracle(h, eri_from_cholesky(L), N, twoS, mps)
    ts = o.two_site(k)
    plan = g.Plan(h, L, K, N, twoS, D, path)
    plan.set_bond(k)
    dim, offs, qn = plan.layout()
    # the canonical layout agrees sector by sector
    assert dim == ts.dim
    lab = [b[0:2] for b in mps.bonds[k - 1]]
    assert len(qn) == len(ts.layout)
    for row, (il, c1, c2, ir, off, dl, dr) in zip(qn, ts.layout):
        assert tuple(row) == (lab[il][0], lab[il][1], c1, c2, dl, dr)
    psi = si.random_vector(dim, seed=1, nvec=nvec).reshape(nvec, dim)
    ref = np.array([ts.sigma(p) for p in psi])
    x = torch.from_numpy(psi.copy()).cuda()
    y = torch.empty_like(x)
    plan.sigma(x, y, nvec=nvec)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    for v in range(nvec):
        assert rel_err(got[v], ref[v]) <= TOL_REL, rel_err(got[v], ref[v])
        assert np.abs(got[v] - ref[v]).max() <= TOL_ELT * np.abs(ref[v]).max()
    d = torch.empty(dim, dtype=torch.float64, device="cuda")
    plan.hdiag(d)
    hd = d.cpu().numpy()
    hd_ref = ts.hdiag()
    assert np.abs(hd - hd_ref).max() <= 1e-11 * np.abs(hd_ref).max()
    st = plan.stats()
    assert st["sigma_flops"] > 0 and st["kernel_launches"] > 0
    plan.close()
    return got


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_sigma_small_truncated_every_bond(tmp_path, k):
    """K=5, N=5, 2Sz=1, D=10: vacuum left block (k=1) and right block (k=4)."""
    _compare_bond(tmp_path, 5, 5, 1, 10, k)


def test_sigma_full_D_middle(tmp_path):
    _compare_bond(tmp_path, 6, 6, 0, 64, 3)


def test_sigma_multi_tile_ragged(tmp_path):
    """K=14, D=600, Gaussian split: sector dims up to 191 (several 64-tiles and a ragged tail)."""
    _compare_bond(tmp_path, 14, 14, 0, 600, 7, split="gaussian", wn=1.0, ws=1.0)


def test_sigma_several_vectors(tmp_path):
    _compare_bond(tmp_path, 8, 8, 0, 40, 4, nvec=3)


def test_sigma_host_buffers_match_device(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    h, L, mps, path = make_case(tmp_path, 8, 8, 0, 40, center=4)
    plan = g.Plan(h, L, 8, 8, 0, 40, path)
    plan.set_bond(4)
    dim = plan.dim
    psi = si.random_vector(dim, seed=3)
    out = np.zeros(dim)
    plan.sigma_host(psi, out)
    x = torch.from_numpy(psi).cuda()
    y = torch.empty_like(x)
    plan.sigma(x, y)
    torch.cuda.synchronize()
    assert np.abs(out - y.cpu().numpy()).max() == 0.0
    plan.close()


def test_sigma_hermitian_gpu(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    h, L, mps, path = make_case(tmp_path, 10, 10, 0, 120, center=5)
    plan = g.Plan(h, L, 10, 10, 0, 120, path)
    plan.set_bond(5)
    dim = plan.dim
    a = torch.from_numpy(si.random_vector(dim, seed=4)).cuda()
    b = torch.from_numpy(si.random_vector(dim, seed=5)).cuda()
    sa, sb = torch.empty_like(a), torch.empty_like(b)
    plan.sigma(a, sa)
    plan.sigma(b, sb)
    x, y = float(a @ sb), float(b @ sa)
    assert abs(x - y) <= 1e-12 * max(1.0, abs(x))
    plan.close()
