"""Extrapolation of DMRG energies to zero discarded weight (oracle).

THIS MODULE IS TEST INFRASTRUCTURE (see the package docstring).

The paper extrapolates the energies E of a series of runs at growing bond
dimension D linearly in their discarded weights w, E(w) = A w + E_{w=0}
(Tab. energy and its caption, Fig. extrapolation).  The oracle is that
straight line fitted by ordinary least squares, written out as the two
normal equations and solved by Cramer's rule; E_{w=0} is the intercept.
"""
import numpy as np


def linear_extrapolation(w, E):
    """Least-squares line E = A w + E0 through the points (w_i, E_i);
    returns (E0, A).  Needs at least two distinct weights."""
    w = np.asarray(w, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    if w.shape != E.shape or w.ndim != 1 or w.size < 2:
        raise ValueError("need two equally long 1-D series of at least two points")
    n = float(w.size)
    sw, sE = w.sum(), E.sum()
    sww, swE = (w * w).sum(), (w * E).sum()
    # normal equations:  [sww sw; sw n] [A; E0] = [swE; sE]
    det = sww * n - sw * sw
    if not det > 0.0:
        raise ValueError("the weights must not all be equal")
    A = (swE * n - sw * sE) / det
    E0 = (sww * sE - sw * swE) / det
    return float(E0), float(A)
