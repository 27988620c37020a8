"""Extrapolation to zero discarded weight over a D schedule run on the GPU
(Tab. energy: energies of sweeps at decreasing D against their largest
discarded weight, fitted by a straight line E(w) = A w + E_{w=0}).

K=8, N=8 (FCI known): dmrg_sweep runs two sweeps at each of D = 48, 32, 24,
16; the last sweep of each D gives one (w, E) point.  dmrg_extrapolate must
agree with the oracle's least-squares line on those points, the energies must
stay variational and fall with D, and E_{w=0} must lie closer to FCI than the
smallest-D energy."""
import os

import numpy as np
import pytest

from oracle.extrapolate import linear_extrapolation
from tests.helpers import cuda_torch, gpu_lib, make_case

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.txt")


def fci_k8():
    for line in open(GOLDEN):
        if line.startswith("k8_n8 "):
            return float(line.split(":")[1].split()[0])
    raise KeyError("k8_n8")


def test_d_schedule_sweeps_extrapolate_like_the_oracle(tmp_path):
    cuda_torch()
    g = gpu_lib()
    K, N = 8, 8
    efci = fci_k8()
    Ds = [48, 32, 24, 16]
    sched = [d for d in Ds for _ in range(2)]
    h, L, mps, path = make_case(tmp_path, K, N, 0, Ds[0], center=1)
    plan = g.Plan(h, L, K, N, 0, Ds[0], path, tol=1e-9)
    e, w = plan.sweep(len(sched), sched)
    plan.close()
    E = e[1::2]
    W = w[1::2]
    print("D", Ds, "E - FCI", E - efci, "w", W)
    assert np.all(E >= efci - 1e-10)
    assert np.all(np.diff(E) > -1e-10)  # smaller D, higher energy
    assert np.all(np.diff(W) > 0.0)     # smaller D, more discarded weight
    e0, a, rms = g.extrapolate(W, E)
    o0, oa = linear_extrapolation(W, E)
    print(f"E(w=0) - FCI = {e0 - efci:.3e}, slope {a:.3f}, rms {rms:.2e}")
    assert abs(e0 - o0) < 1e-9 and abs(a - oa) < 1e-7 * max(1.0, abs(oa))
    assert abs(e0 - efci) < abs(E[-1] - efci)
