"""Test helpers: node coordinates and manufactured data built from the oracle's tables
(never from the GPU library), so that every input the parity tests feed to both sides
comes from the oracle or from ``synthetic``."""
import numpy as np

from oracle.points import boundary_points, leaf_points  # noqa: F401  (re-exported)


def poly_data(X, Y, coeffs, a, b):
    """u = x^a y^b and g = A u evaluated in closed form (Eq. defA)."""
    def mono(i, j, dx, dy):
        cx = 1.0
        for k in range(dx):
            cx *= (i - k)
        cy = 1.0
        for k in range(dy):
            cy *= (j - k)
        if cx == 0.0 or cy == 0.0:
            return np.zeros_like(X)
        return cx * cy * X ** (i - dx) * Y ** (j - dy)
    u = mono(a, b, 0, 0)
    c11, c12, c22, c1, c2, c0 = coeffs
    g = (-c11 * mono(a, b, 2, 0) - 2 * c12 * mono(a, b, 1, 1) - c22 * mono(a, b, 0, 2)
         + c1 * mono(a, b, 1, 0) + c2 * mono(a, b, 0, 1) + c0 * u)
    return u, g


def rel_linf(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))
