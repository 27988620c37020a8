"""Argument and input checks of dmrg_plan that return before any device work
(host logic, no GPU): non-finite integrals give DMRG_ENUMERIC, quantum numbers
that do not fit K give DMRG_EINVAL, a missing MPS path gives DMRG_EINVAL."""
import numpy as np
import pytest

import synthetic_inputs as si


def _lib():
    import paper_2311_02854_gb300 as g
    try:
        g.lib()
    except (RuntimeError, OSError) as e:  # the library is built by build()
        pytest.skip(f"libdmrg.so not available: {e}")
    return g


def test_non_finite_integrals_are_rejected(tmp_path):
    g = _lib()
    h, L = si.make_integrals(4, 8, seed=0)
    for bad in (np.nan, np.inf):
        h2 = h.copy()
        h2[1, 2] = bad
        with pytest.raises(g.DMRGError) as e:
            g.Plan(h2, L, 4, 4, 0, 16, str(tmp_path / "none.bin"))
        assert e.value.code == -4
        L2 = L.copy()
        L2[3, 0, 1] = bad
        with pytest.raises(g.DMRGError) as e:
            g.Plan(h, L2, 4, 4, 0, 16, str(tmp_path / "none.bin"))
        assert e.value.code == -4


@pytest.mark.parametrize("N,twoS", [(9, 0), (4, 1), (4, 6), (-1, 1)])
def test_inconsistent_quantum_numbers_are_rejected(tmp_path, N, twoS):
    g = _lib()
    h, L = si.make_integrals(4, 8, seed=0)
    with pytest.raises(g.DMRGError) as e:
        g.Plan(h, L, 4, N, twoS, 16, str(tmp_path / "none.bin"))
    assert e.value.code == -1
