"""dmrg_extrapolate (host arithmetic in the library, no GPU) against the
oracle's least-squares extrapolation: the paper's Tab. energy series and
seeded series; degenerate inputs are rejected with DMRG_EINVAL."""
import numpy as np
import pytest

import paper_2311_02854_gb300 as g
from oracle.extrapolate import linear_extrapolation
from tests.test_oracle_extrapolate import tab_energy


def test_library_matches_the_oracle_on_the_paper_series():
    for name, (e0_ref, D, w, E) in tab_energy().items():
        e0, a, rms = g.extrapolate(w, E)
        o0, oa = linear_extrapolation(w, E)
        # two algebraic routes (centred moments vs normal equations) in FP64
        assert abs(e0 - o0) < 1e-8 and abs(a - oa) < 1e-6 * abs(oa)
        assert abs(e0 - e0_ref) < 1e-5 and 0.0 < rms < 1e-3


def test_library_matches_the_oracle_on_seeded_series():
    rng = np.random.default_rng(7)
    for n in (2, 3, 10, 100):
        w = rng.uniform(1e-6, 1e-3, n)
        E = -2000.0 + rng.uniform(50, 300) * w + rng.normal(0, 1e-6, n)
        e0, a, rms = g.extrapolate(w, E)
        o0, oa = linear_extrapolation(w, E)
        assert abs(e0 - o0) < 1e-9 * 2000.0 and abs(a - oa) < 1e-7 * max(1.0, abs(oa))
        resid = E - (oa * w + o0)
        assert abs(rms - np.sqrt(np.mean(resid ** 2))) < 1e-9


@pytest.mark.parametrize("w,E", [([1e-4], [-1.0]), ([2e-4, 2e-4], [-1.0, -1.1]), ([1e-4, np.nan], [-1.0, -2.0])])
def test_degenerate_series_are_rejected(w, E):
    with pytest.raises(g.DMRGError) as exc:
        g.extrapolate(w, E)
    assert exc.value.code == -1
