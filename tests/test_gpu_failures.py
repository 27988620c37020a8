"""Failure detection on the GPU path, made on the host (no kernel is made to
fault or hang): a non-finite guess is caught by Davidson's FP64 norm check
(DMRG_ENUMERIC), a device budget smaller than the plan needs is refused before
the allocation (DMRG_ENOMEM), an unreadable MPS file gives DMRG_EIO; the
context stays usable after each."""
import numpy as np
import pytest

import synthetic_inputs as si
from tests.helpers import cuda_torch, gpu_lib, make_case

pytestmark = pytest.mark.gpu


def test_nan_guess_gives_enumeric(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 6, 6, 0, 20, 3
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    for prec in (0, 1):
        plan = g.Plan(h, L, K, N, twoS, D, path, precision=prec)
        plan.set_bond(k)
        psi = si.random_vector(plan.dim, seed=1)
        psi[plan.dim // 2] = np.nan
        x = torch.from_numpy(psi).cuda()
        with pytest.raises(g.DMRGError) as e:
            plan.davidson(x, 1, tol=1e-8, max_iter=50)
        assert e.value.code == -4
        # the plan still works with a finite guess
        x = torch.from_numpy(si.random_vector(plan.dim, seed=1)).cuda()
        en, it, conv = plan.davidson(x, 1, tol=1e-6, max_iter=200)
        assert np.isfinite(en[0])
        plan.close()


def test_budget_too_small_gives_enomem(tmp_path):
    torch = cuda_torch()
    g = gpu_lib()
    K, N, twoS, D, k = 8, 8, 0, 64, 4
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(g.DMRGError) as e:
        plan = g.Plan(h, L, K, N, twoS, D, path, mem_budget=200 << 10)
        try:
            plan.set_bond(k)
        finally:
            plan.close()
    assert e.value.code == -2 and "budget" in str(e.value)
    torch.cuda.synchronize()
    # nothing stays allocated, and a plan with enough budget runs
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    plan = g.Plan(h, L, K, N, twoS, D, path)
    plan.set_bond(k)
    plan.close()


def test_unreadable_mps_file_gives_eio(tmp_path):
    cuda_torch()
    g = gpu_lib()
    h, L = si.make_integrals(6, 24, seed=0)
    with pytest.raises(g.DMRGError) as e:
        g.Plan(h, L, 6, 6, 0, 20, str(tmp_path / "missing.bin"))
    assert e.value.code == -7
    bad = tmp_path / "truncated.bin"
    bad.write_bytes(b"\x00\x01\x02")
    with pytest.raises(g.DMRGError) as e:
        g.Plan(h, L, 6, 6, 0, 20, str(bad))
    assert e.value.code in (-7, -1)


def test_bounded_wait_gives_etimeout_and_the_context_stays_usable(tmp_path):
    """A wait on an mbarrier that nothing arrives on (the wait routine of the
    tensor-core kernels, with a 0.2 s limit) gives up and reports
    DMRG_ETIMEOUT; the same wait with an arrival completes, and a sigma runs
    afterwards."""
    torch = cuda_torch()
    g = gpu_lib()
    with pytest.raises(g.DMRGError) as e:
        g.selftest_wait(0.2, arrive=False)
    assert e.value.code == -5
    g.selftest_wait(0.2, arrive=True)
    with pytest.raises(g.DMRGError) as e:
        g.selftest_wait(3.0, arrive=True)
    assert e.value.code == -1
    K, N, twoS, D, k = 6, 6, 0, 20, 3
    h, L, mps, path = make_case(tmp_path, K, N, twoS, D, center=k)
    plan = g.Plan(h, L, K, N, twoS, D, path, precision=1)
    plan.set_bond(k)
    x = torch.from_numpy(si.random_vector(plan.dim, seed=1)).cuda()
    y = torch.empty_like(x)
    plan.sigma(x, y)
    assert np.isfinite(y.cpu().numpy()).all()
    plan.close()
