"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/dmrg.h (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dmrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(dmrg_[A-Za-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["dmrg_plan", "dmrg_set_bond", "dmrg_layout", "dmrg_sigma", "dmrg_davidson", "dmrg_sweep",
              "dmrg_save_mps", "dmrg_stats", "dmrg_last_error", "dmrg_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2311_02854_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_plan_arguments():
    import numpy as np
    import paper_2311_02854_gb300 as g
    with pytest.raises(g.DMRGError):
        g.Plan(np.zeros((2, 2)), np.zeros((1, 2, 2)), 2, 9, 0, 4, "/nonexistent")
