"""Tile shapes of the mixed sigma: both tile widths and both phase-2 K-chunks
against the FP64 oracle, and the autotuner that picks among them per sector-size
histogram (its choice, its timings and its cache)."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle.dmrg import Oracle
from oracle.hamiltonian import eri_from_cholesky
from tests.helpers import cuda_torch, gpu_lib, make_case, rel_err

pytestmark = pytest.mark.gpu

BF16X3 = 1
CASE = dict(K=14, N=14, twoS=0, D=600, k=7)


def _case(tmp_path):
    c = CASE
    h, L, mps, path = make_case(tmp_path, c["K"], c["N"], c["twoS"], c["D"], center=c["k"], split="gaussian",
                                wn=1.0, ws=1.0)
    ts = Oracle(h, eri_from_cholesky(L), c["N"], c["twoS"], mps).two_site(c["k"])
    return h, L, path, ts


def _sigma(plan, psi):
    torch = cuda_torch()
    x = torch.from_numpy(psi.copy()).cuda()
    y = torch.empty_like(x)
    plan.sigma(x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("tile_n,kchunk", [(64, 0), (128, 512), (64, 512)])
def test_fixed_tile_shapes_match_oracle(tmp_path, tile_n, kchunk):
    g = gpu_lib()
    h, L, path, ts = _case(tmp_path)
    c = CASE
    plan = g.Plan(h, L, c["K"], c["N"], c["twoS"], c["D"], path, precision=BF16X3, sigma_tile_n=tile_n,
                  tc_kchunk=kchunk)
    plan.set_bond(c["k"])
    st = plan.stats()
    assert st["sigma_tile_n"] == tile_n and st["tunes"] == 0
    assert st["sigma_kchunk"] == (kchunk if kchunk else 1024)
    psi = si.random_vector(plan.dim, seed=1)
    err = rel_err(_sigma(plan, psi), ts.sigma(psi))
    print(f"tile {tile_n} kchunk {st['sigma_kchunk']}: sigma vs oracle {err:.2e}, tiles {st['sigma_tiles']}")
    assert err <= 2e-5
    plan.close()


def test_autotuner_choice_timings_and_cache(tmp_path):
    g = gpu_lib()
    h, L, path, ts = _case(tmp_path)
    c = CASE
    plan = g.Plan(h, L, c["K"], c["N"], c["twoS"], c["D"], path, precision=BF16X3)
    plan.set_bond(c["k"])
    st = plan.stats()
    assert st["tunes"] == 1 and st["tune_hits"] == 0
    cand = st["tune_cand_ms"]
    assert all(t > 0.0 for t in cand)
    shapes = [(128, 1024), (64, 1024), (128, 512), (64, 512)]
    chosen = (st["sigma_tile_n"], st["sigma_kchunk"])
    assert chosen in shapes
    # the default unless another candidate was at least 2 % faster; never a slower one
    i = shapes.index(chosen)
    assert cand[i] == min(cand) or (i == 0 and min(cand) >= 0.98 * cand[0])
    print(f"candidates (ms): {cand}, chosen {chosen}, tuning {st['ms_tune']:.0f} ms")
    psi = si.random_vector(plan.dim, seed=1)
    ref = ts.sigma(psi)
    assert rel_err(_sigma(plan, psi), ref) <= 2e-5
    # same bond again: same histogram, the cached choice, no new tuning
    plan.set_bond(c["k"])
    st2 = plan.stats()
    assert st2["tunes"] == 1 and st2["tune_hits"] == 1
    assert (st2["sigma_tile_n"], st2["sigma_kchunk"]) == chosen
    assert rel_err(_sigma(plan, psi), ref) <= 2e-5
    plan.close()


def test_bad_tile_width_is_rejected(tmp_path):
    g = gpu_lib()
    h, L, path, ts = _case(tmp_path)
    c = CASE
    with pytest.raises(g.DMRGError):
        g.Plan(h, L, c["K"], c["N"], c["twoS"], c["D"], path, precision=BF16X3, sigma_tile_n=96)
