"""Pins of the oracle on indefinite (Helmholtz) operators, c < 0 (Sec. 7.2): exact plane
waves are reproduced to spectral accuracy, the error falls with p, and the variable-
coefficient scattering problem agrees with the dense global collocation solve."""
import numpy as np

import synthetic as syn
from oracle import dense, hps, tree as tr
from tests.helpers import boundary_points, leaf_points


def _plane_wave_error(n, p, kappa):
    t = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(t, p)
    bx, by = boundary_points(t)
    z = np.zeros_like(X)
    coeffs = np.array([z + 1, z, z + 1, z, z, z - kappa ** 2])
    u, _ = hps.solve(t, hps.build(t, coeffs, p), p, syn.plane_wave(bx, by, kappa), np.zeros_like(X))
    return np.max(np.abs(u[..., 0] - syn.plane_wave(X, Y, kappa)))


def test_plane_wave_kappa20():
    # -Laplace(u) - 400 u = 0 with u a plane wave: closed form, g = 0
    assert _plane_wave_error(4, 16, 20.0) < 1e-9


def test_plane_wave_error_falls_with_p():
    e = [_plane_wave_error(2, p, 20.0) for p in (8, 12, 16)]
    assert e[0] > 10 * e[1] > 100 * e[2]


def test_scattering_problem_matches_dense_solve():
    n, p = 2, 10
    t = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(t, p)
    bx, by = boundary_points(t)
    c, g = syn.helmholtz_scattering(X, Y, kappa=10.0)
    coeffs = np.array(c)
    assert np.min(coeffs[5]) < -50.0
    f = np.zeros_like(bx)
    u, _ = hps.solve(t, hps.build(t, coeffs, p), p, f, g)
    ud, _ = dense.solve(t, coeffs, p, f, g)
    assert np.max(np.abs(u - ud)) < 1e-10 * np.max(np.abs(ud))
