"""Pins for the oracle adjoint (transposed Algorithm 2 sweeps and coefficient gradients):
the dot-product identity, the brute-force transposed solve, and central finite differences."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dense, hps, spectral as sp, tree as tr
from tests.helpers import boundary_points, leaf_points


def _setup(nx=2, ny=2, p=8):
    t = tr.uniform_tree(0, 0, 1, 1, nx, ny, p - 1)
    X, Y = leaf_points(t, p)
    prob = syn.VarCoeffProblem()
    coeffs = np.array(prob.coeffs(X, Y))
    bx, by = boundary_points(t)
    return t, coeffs, prob.load(X, Y), prob.dirichlet(bx, by), X, Y


def test_dot_product_identity():
    # <Sol(f, g, rho), ubar> = <f, fbar> + <g, gbar> + <rho, rhobar>
    p = 8
    t, coeffs, _, _, _, _ = _setup(3, 2, p)
    ops = hps.build(t, coeffs, p)
    rng = np.random.default_rng(11)
    f = rng.standard_normal((len(t.boundary), 2))
    g = rng.standard_normal((t.n_leaves, p * p, 2))
    rho = rng.standard_normal((t.n_gauss, 2))
    rho[t.boundary] = 0.0
    ubar = rng.standard_normal((t.n_leaves, p * p, 2))
    uc, _ = hps.solve(t, ops, p, f, g, rho)
    fb, gb, rb = hps.adjoint(t, ops, p, ubar)
    lhs = np.sum(uc * ubar)
    _, ci, _ = sp.leaf_index_sets(p)
    rhs = np.sum(f * fb) + np.sum(g[:, ci] * gb[:, ci]) + np.sum(rho * rb)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    ce, _, _ = sp.leaf_index_sets(p)
    assert np.all(gb[:, ce] == 0.0)


@pytest.mark.parametrize("nx,ny,p", [(1, 1, 7), (2, 2, 8), (3, 1, 6)])
def test_matches_dense_transpose(nx, ny, p):
    t, coeffs, _, _, _, _ = _setup(nx, ny, p)
    ops = hps.build(t, coeffs, p)
    ubar = np.random.default_rng(7).standard_normal((t.n_leaves, p * p, 1))
    fb, gb, rb = hps.adjoint(t, ops, p, ubar)
    fd, gd, rd = dense.solve_transpose(t, coeffs, p, ubar)
    scale = max(np.max(np.abs(gd)), np.max(np.abs(fd)))
    assert np.max(np.abs(fb - fd)) < 1e-10 * scale
    assert np.max(np.abs(gb - gd)) < 1e-10 * scale
    assert np.max(np.abs(rb - rd)) < 1e-10 * scale


def test_gradients_central_differences():
    # Gradients of J = 0.5 ||u - u_obs||^2 w.r.t. every coefficient field and g, checked
    # along seeded random directions by central differences with h = 1e-6 (rebuild each time).
    p = 8
    t, coeffs, g, f, X, Y = _setup(2, 2, p)
    prob = syn.VarCoeffProblem()
    obs_coeffs = np.array(prob.coeffs(X, Y, perturbed=True))
    u_obs = hps.solve(t, hps.build(t, obs_coeffs, p), p, f, g)[0]

    def J(cf, gg):
        u = hps.solve(t, hps.build(t, cf, p), p, f, gg)[0]
        return 0.5 * np.sum((u - u_obs) ** 2)

    ops = hps.build(t, coeffs, p)
    u = hps.solve(t, ops, p, f, g)[0]
    fb, gb, _ = hps.adjoint(t, ops, p, u - u_obs)
    grads = hps.coeff_gradients(t, p, u, gb)
    h = 1e-6
    dirs = syn.random_directions(coeffs.shape, n=3)
    for v in dirs:
        fd = (J(coeffs + h * v, g) - J(coeffs - h * v, g)) / (2 * h)
        an = np.sum(grads * v)
        assert abs(fd - an) < 1e-5 * max(abs(an), 1e-12)
    vg = syn.random_directions(g.shape, n=1, seed_offset=900)[0]
    fd = (J(coeffs, g + h * vg) - J(coeffs, g - h * vg)) / (2 * h)
    an = np.sum(gb[..., 0] * vg)
    assert abs(fd - an) < 1e-5 * abs(an)


def test_reaction_gradient_identity():
    # dJ/dc = -gbar * u at interior nodes: perturbing c at one interior node of one leaf.
    p = 7
    t, coeffs, g, f, _, _ = _setup(2, 1, p)
    ops = hps.build(t, coeffs, p)
    u = hps.solve(t, ops, p, f, g)[0]
    target = np.zeros_like(u)
    _, gb, _ = hps.adjoint(t, ops, p, u - target)
    _, ci, _ = sp.leaf_index_sets(p)
    lf, node = 1, ci[5]
    h = 1e-6
    vals = []
    for s in (1, -1):
        cf = coeffs.copy()
        cf[5, lf, node] += s * h
        uu = hps.solve(t, hps.build(t, cf, p), p, f, g)[0]
        vals.append(0.5 * np.sum(uu ** 2))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - (-gb[lf, node, 0] * u[lf, node, 0])) < 1e-6 * abs(fd)
