"""The oracle's linear extrapolation E(w) = A w + E_{w=0} against the paper's
printed example (Tab. energy) and against what the mathematics fixes."""
import os

import numpy as np
import pytest

from oracle.extrapolate import linear_extrapolation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tab_energy_extrapolation.txt")


def tab_energy():
    """{series: (E_w0 printed, D, w, E)} from the golden file."""
    out, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "series":
            cur = f[1]
            out[cur] = (float(f[2]), [], [], [])
        else:
            out[cur][1].append(int(f[0]))
            out[cur][2].append(float(f[1]))
            out[cur][3].append(float(f[2]))
    return out


def test_reproduces_the_printed_extrapolations():
    """All points of each column fitted by least squares give the printed
    E_{w=0}: to 1e-6 Eh for the two series whose weights are printed with
    enough digits, to 1e-5 Eh for the paper's own series, whose weights carry
    three significant digits (a rounding of 5e-8 in w moves E_{w=0} by up
    to |A| x 5e-8 ~ 1e-5 Eh with A ~ 170 Eh)."""
    tab = tab_energy()
    assert set(tab) == {"li2019", "lee2023", "this_work"}
    for name, tol in (("li2019", 1e-6), ("lee2023", 1e-6), ("this_work", 1e-5)):
        e0_ref, D, w, E = tab[name]
        e0, a = linear_extrapolation(w, E)
        assert abs(e0 - e0_ref) <= tol, (name, e0, e0_ref)
        assert a > 0.0  # the energy rises with the discarded weight


def test_exact_line_and_invariances():
    rng = np.random.default_rng(5)
    w = rng.uniform(1e-6, 1e-3, 12)
    E = 173.25 * w - 17492.5
    e0, a = linear_extrapolation(w, E)
    assert abs(e0 + 17492.5) < 1e-9 and abs(a - 173.25) < 1e-6
    # the order of the points does not matter
    p = rng.permutation(w.size)
    e0p, ap = linear_extrapolation(w[p], E[p])
    assert abs(e0p - e0) < 1e-9 and abs(ap - a) < 1e-6
    # two points: the line through them
    e0, a = linear_extrapolation([1e-4, 3e-4], [-1.0, -0.5])
    assert abs(a - 2500.0) < 1e-9 and abs(e0 + 1.25) < 1e-12


def test_against_a_library_fit_with_noise():
    rng = np.random.default_rng(6)
    w = rng.uniform(1e-5, 5e-4, 20)
    E = -100.0 + 80.0 * w + rng.normal(0.0, 1e-5, w.size)
    e0, a = linear_extrapolation(w, E)
    a_np, e0_np = np.polyfit(w, E, 1)
    assert abs(e0 - e0_np) < 1e-9 and abs(a - a_np) < 1e-4


@pytest.mark.parametrize("w,E", [([1e-4], [-1.0]), ([2e-4, 2e-4], [-1.0, -1.1]), ([1e-4, 2e-4], [-1.0])])
def test_degenerate_series_are_rejected(w, E):
    with pytest.raises(ValueError):
        linear_extrapolation(w, E)
