"""Shared test helpers: seeded problem construction (inputs only)."""
import os

import numpy as np
import pytest

import synthetic_inputs as si


def cuda_torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_lib():
    import paper_2311_02854_gb300 as g
    g.lib()  # fails loudly if the extension is missing
    return g


def make_case(tmpdir, K, N, twoS, D, center, split="proportional", wn=None, ws=None, n_chol=None,
              ell=3.0, h_min=-4.0, seed_mps=2):
    h, L = si.make_integrals(K, n_chol or 4 * K, ell=ell, h_min=h_min, seed=0)
    bonds = si.bond_sectors(K, N, twoS, D, split, wn, ws)
    mps = si.random_mps(K, N, twoS, bonds, center=center, seed=seed_mps)
    path = os.path.join(str(tmpdir), f"mps_{K}_{N}_{twoS}_{D}_{center}_{split}.bin")
    si.write_mps(path, mps)
    return h, L, mps, path


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
