"""Host tier of the environment blocks during sweeps (Sec. 2.3: operators of
the blocks away from the current bond are kept off the GPU).

A sweep with the tier must give the energies and discarded weights of the
same sweep without it (the same arithmetic on blocks that made a round trip
through pinned host memory), move blocks both ways, and hold less device
memory at its high-water mark.  FP64 sweeps are deterministic and must agree
bitwise; the FP64-accurate tensor-core engine sums some tiles with atomics
(order-dependent rounding near 1e-15 relative); BF16X3 sweeps differ from run
to run at the mixed sigma's noise floor (order of the FP64 atomics of the
drains, amplified by a Davidson that stops at that floor), so they are held to
that floor only."""
import numpy as np
import pytest

from tests.helpers import cuda_torch, gpu_lib, make_case

pytestmark = pytest.mark.gpu


def _sweeps(g, tmp_path, precision, tier, K=12, N=12, D=160, n=2):
    h, L, mps, path = make_case(tmp_path, K, N, 0, D, center=1)
    plan = g.Plan(h, L, K, N, 0, D, path, tol=1e-8, precision=precision, host_tier=tier, sigma_tune=0)
    e, w = plan.sweep(n)
    st = plan.stats()
    plan.close()
    return e, w, st


@pytest.mark.parametrize("precision,tol", [(0, 0.0), (4, 1e-9), (1, 1e-3)])
def test_host_tier_sweep_matches_resident_sweep(tmp_path, precision, tol):
    cuda_torch()
    g = gpu_lib()
    e0, w0, s0 = _sweeps(g, tmp_path, precision, 0)
    e1, w1, s1 = _sweeps(g, tmp_path, precision, 1)
    print(f"precision {precision}: E {e0[-1]:.12f} / {e1[-1]:.12f}, peak device "
          f"{s0['device_bytes_peak'] / 2**20:.1f} / {s1['device_bytes_peak'] / 2**20:.1f} MiB, "
          f"out {s1['tier_out_bytes'] / 2**20:.1f} MiB, in {s1['tier_in_bytes'] / 2**20:.1f} MiB, "
          f"pinned {s1['host_bytes'] / 2**20:.1f} MiB, wait {s1['ms_tier_wait']:.1f} ms")
    assert np.max(np.abs(e1 - e0)) <= tol
    assert np.max(np.abs(w1 - w0)) <= max(tol, 1e-12 if precision else 0.0)
    assert s0["tier_out_bytes"] == 0 and s0["tier_in_bytes"] == 0 and s0["host_bytes"] == 0
    assert s1["tier_out_bytes"] > 0 and s1["tier_in_bytes"] > 0 and s1["host_bytes"] > 0
    assert s1["device_bytes_peak"] < s0["device_bytes_peak"]


def test_host_tier_every_block_comes_back(tmp_path):
    """Three sweeps: the second and third read right / left blocks that spent
    the previous half-sweep on the host; the energy of the last sweep equals
    the resident run's."""
    cuda_torch()
    g = gpu_lib()
    e0, _, _ = _sweeps(g, tmp_path, 0, 0, K=10, N=10, D=100, n=3)
    e1, _, s1 = _sweeps(g, tmp_path, 0, 1, K=10, N=10, D=100, n=3)
    assert np.max(np.abs(e1 - e0)) == 0.0
    # each block is copied out once; the blocks of the last half sweep never come back
    assert 0 < s1["tier_in_bytes"] <= s1["tier_out_bytes"]
