"""Pins for the oracle's local refinement (Sec. 6) and union-of-squares domains:
polynomial exactness, the brute-force system with coarse-fine interface equations, the
adjoint, interpolation exactness of P_up / P_down, the paper's leaf count and the
re-entrant-corner solution on the L-shaped domain."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dense, hps, tree as tr
from tests.helpers import boundary_points, leaf_points, poly_data, rel_linf

CASES = [((3, 3), [(0.1, 0.9)], 2, 6), ((2, 2), [(0.3, 0.3)], 2, 7), ((6, 3), [(0.6, 0.2), (0.05, 0.95)], 1, 6),
         ((4, 2), [(0.6, 0.1)], 2, 5)]


def _refined(base, pts, lev, p):
    return tr.refine_tree(tr.uniform_tree(0, 0, 1, 1, base[0], base[1], p - 1), pts, lev)


def _coeffs(t, p):
    X, Y = leaf_points(t, p)
    prob = syn.VarCoeffProblem()
    return np.array(prob.coeffs(X, Y)), prob, X, Y


@pytest.mark.parametrize("base,pts,lev,p", CASES)
def test_refined_polynomial_exactness(base, pts, lev, p):
    t = _refined(base, pts, lev, p)
    assert any(b.Pup is not None for b in t.boxes)  # the case has coarse-fine interfaces
    coeffs, _, X, Y = _coeffs(t, p)
    ops = hps.build(t, coeffs, p)
    bx, by = boundary_points(t)
    for a, b in [(0, 0), (1, 3), (p - 2, 2)]:
        u, g = poly_data(X, Y, coeffs, a, b)
        uc, _ = hps.solve(t, ops, p, bx ** a * by ** b, g)
        assert np.max(np.abs(uc[..., 0] - u)) < 1e-10


@pytest.mark.parametrize("base,pts,lev,p", CASES)
def test_refined_matches_brute_force_and_adjoint(base, pts, lev, p):
    t = _refined(base, pts, lev, p)
    coeffs, prob, X, Y = _coeffs(t, p)
    bx, by = boundary_points(t)
    g, f = prob.load(X, Y), prob.dirichlet(bx, by)
    rho = np.random.default_rng(8).standard_normal(t.n_gauss)
    ops = hps.build(t, coeffs, p)
    uc, ug = hps.solve(t, ops, p, f, g, rho)
    ucd, ugd = dense.solve(t, coeffs, p, f, g, rho)
    assert rel_linf(uc, ucd) < 1e-10 and rel_linf(ug, ugd) < 1e-10
    ubar = np.random.default_rng(9).standard_normal(uc.shape)
    fb, gb, rb = hps.adjoint(t, ops, p, ubar)
    fd, gd, rd = dense.solve_transpose(t, coeffs, p, ubar)
    sc = max(np.max(np.abs(gd)), np.max(np.abs(fd)))
    assert np.max(np.abs(gb - gd)) < 1e-10 * sc and np.max(np.abs(fb - fd)) < 1e-10 * sc
    assert np.max(np.abs(rb - rd)) < 1e-10 * sc


def test_interpolation_operators_exact_on_polynomials():
    # P_up (coarse -> fine) and P_down (fine -> coarse) reproduce polynomials of degree <= q-1
    # along each side, including coarse nodes on the boundary between two fine segments (odd q).
    for q in (5, 6):
        t = _refined((4, 4), [(0.37, 0.58)], 2, q + 1)
        xy = t.gauss_points()
        checked = 0
        for b in t.boxes:
            if b.Pup is None:
                continue
            for deg in (0, 1, q - 1):
                fun = lambda P: (P[:, 0] + 0.3 * P[:, 1]) ** deg
                assert np.max(np.abs(b.Pup @ fun(xy[b.ge]) - fun(xy[b.ge_old]))) < 1e-11
                assert np.max(np.abs(b.Pdown @ fun(xy[b.ge_old]) - fun(xy[b.ge]))) < 1e-11
            checked += 1
        assert checked > 0


def test_refined_leaf_count_matches_paper():
    # Sec. 7.3: 4 x 4 leaves with one level of refinement at the centre give 28 leaves.
    t = tr.refine_tree(tr.uniform_tree(0, 0, 1, 1, 4, 4, 6), [(0.5, 0.5)], 1)
    assert t.n_leaves == 28


def test_l_shape_polynomial_and_brute_force():
    p = 7
    t = tr.refine_tree(tr.l_shape_tree(2, p - 1), [(0.0, 0.0)], 2)
    coeffs, prob, X, Y = _coeffs(t, p)
    bx, by = boundary_points(t)
    ops = hps.build(t, coeffs, p)
    u, g = poly_data(X, Y, coeffs, 3, 4)
    uc, _ = hps.solve(t, ops, p, bx ** 3 * by ** 4, g)
    assert np.max(np.abs(uc[..., 0] - u)) < 1e-10
    g, f = prob.load(X, Y), prob.dirichlet(bx, by)
    assert rel_linf(hps.solve(t, ops, p, f, g)[0], dense.solve(t, coeffs, p, f, g)[0]) < 1e-10


def corner_solution(x, y):
    """u = r^(2/3) sin(2 theta / 3), theta in [0, 3 pi / 2] from the edge y = 0, x > 0: the
    harmonic function vanishing on both edges of the re-entrant corner of the L."""
    th = np.mod(np.arctan2(y, x), 2 * np.pi)
    return np.hypot(x, y) ** (2.0 / 3.0) * np.sin(2.0 * th / 3.0)


def test_l_shape_corner_singularity_error_falls_with_refinement():
    # Pin P10 (qualitative, cf. Sec. 7.5): refining toward the re-entrant corner reduces the
    # error of the Laplace solution u = r^(2/3) sin(2 theta / 3).
    p = 10
    errs = []
    for lev in (0, 2, 4):
        t = tr.refine_tree(tr.l_shape_tree(1, p - 1), [(0.0, 0.0)], lev)
        X, Y = leaf_points(t, p)
        n = X.shape
        coeffs = np.array([np.ones(n), np.zeros(n), np.ones(n), np.zeros(n), np.zeros(n), np.zeros(n)])
        bx, by = boundary_points(t)
        uc, _ = hps.solve(t, hps.build(t, coeffs, p), p, corner_solution(bx, by), np.zeros(n))
        errs.append(np.max(np.abs(uc[..., 0] - corner_solution(X, Y))))
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1]
