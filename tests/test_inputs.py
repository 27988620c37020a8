"""The seeded synthetic inputs follow the paper's workload shape: at K = 73,
N = 114 the Gaussian sector split of the benchmark puts the largest
middle-bond sector where the paper's fit of the maximal sector dimension,
d_max(D) = 0.128 D + 51.8 (Eq. dmax, Sec. 3 "Results", fitted to the
sector maxima of Tab. speedup), puts it."""
import pytest

import synthetic_inputs as si


@pytest.mark.parametrize("D", [2000, 3000])
def test_middle_bond_sector_maximum_follows_eq_dmax(D):
    bonds = si.bond_sectors(73, 114, 0, D, "gaussian", 1.45, 1.45)
    mid = bonds[36]
    dims = [s[2] for s in mid]
    assert sum(dims) == D
    dmax = 0.128 * D + 51.8
    assert abs(max(dims) - dmax) <= 0.05 * dmax, (max(dims), dmax)


def test_inputs_are_seeded():
    a = si.make_integrals(8, 32, ell=3.0, h_min=-4.0, seed=0)
    b = si.make_integrals(8, 32, ell=3.0, h_min=-4.0, seed=0)
    assert all((x == y).all() for x, y in zip(a, b))
    assert (si.random_vector(100, seed=1) == si.random_vector(100, seed=1)).all()
