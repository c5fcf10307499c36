"""Pins for the oracle's leaf operators, merges, Algorithms 1-2 and the residual:
polynomial exactness, brute force, spectral convergence, tree-order independence,
DtN identities, flux continuity and heat-equation eigenmodes."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dense, hps, leaf as lfm, spectral as sp, tree as tr
from tests.helpers import boundary_points, leaf_points, poly_data, rel_linf


def _problem(t, p, kind="var"):
    X, Y = leaf_points(t, p)
    if kind == "var":
        prob = syn.VarCoeffProblem()
        coeffs = np.array(prob.coeffs(X, Y))
        bx, by = boundary_points(t)
        return coeffs, prob.load(X, Y), prob.dirichlet(bx, by), (X, Y)
    coeffs, g = syn.poisson_manufactured(X, Y)
    bx, by = boundary_points(t)
    return np.array(coeffs), g, syn.u_star(bx, by), (X, Y)


@pytest.mark.parametrize("nx,ny,p", [(1, 1, 8), (2, 1, 8), (3, 2, 7), (4, 4, 10)])
def test_polynomial_exactness(nx, ny, p):
    # Pin P1: u = x^a y^b with a, b <= q-1 solves the discrete system exactly (every
    # interpolation, differentiation and collocation step is exact for it).
    q = p - 1
    t = tr.uniform_tree(0.1, -0.2, 0.9, 0.7, nx, ny, q)
    coeffs, _, _, (X, Y) = _problem(t, p)
    ops = hps.build(t, coeffs, p)
    bx, by = boundary_points(t)
    for a, b in [(0, 0), (1, 2), (q - 1, 3), (2, q - 1)]:
        u, g = poly_data(X, Y, coeffs, a, b)
        uc, _ = hps.solve(t, ops, p, bx ** a * by ** b, g)
        assert np.max(np.abs(uc[..., 0] - u)) < 1e-10 * max(1.0, np.max(np.abs(u)))


@pytest.mark.parametrize("nx,ny,p", [(1, 1, 6), (2, 1, 7), (1, 2, 8), (2, 2, 9), (3, 3, 6)])
def test_matches_brute_force(nx, ny, p):
    # Pin P2: Algorithms 1-2 eliminate the global collocation system exactly.
    t = tr.uniform_tree(0, 0, 1, 1, nx, ny, p - 1)
    coeffs, g, f, _ = _problem(t, p)
    rng = np.random.default_rng(3)
    rho = rng.standard_normal(t.n_gauss)
    ops = hps.build(t, coeffs, p)
    for r in (None, rho):
        uc, ug = hps.solve(t, ops, p, f, g, r)
        ucd, ugd = dense.solve(t, coeffs, p, f, g, r)
        assert rel_linf(uc, ucd) < 1e-11
        assert rel_linf(ug, ugd) < 1e-11


def test_spectral_convergence_poisson():
    # Pin P3: config-1 style manufactured solution; the error against the closed form
    # falls geometrically with p.
    errs = []
    for p in (6, 8, 10, 12, 14, 16):
        t = tr.uniform_tree(0, 0, 1, 1, 2, 2, p - 1)
        coeffs, g, f, (X, Y) = _problem(t, p, "poisson")
        uc, _ = hps.solve(t, hps.build(t, coeffs, p), p, f, g)
        errs.append(np.max(np.abs(uc[..., 0] - syn.u_star(X, Y))))
    assert errs[-1] < 1e-10
    assert all(errs[k + 1] < 0.2 * errs[k] for k in range(3))


def test_tree_order_independence():
    # Pin P4: vertical-first and horizontal-first splitting solve the same discrete system.
    p = 8
    outs = []
    for tie in ("v", "h"):
        t = tr.uniform_tree(0, 0, 1, 1, 4, 4, p - 1, tie=tie)
        coeffs, g, f, _ = _problem(t, p)
        outs.append(hps.solve(t, hps.build(t, coeffs, p), p, f, g)[0])
    assert rel_linf(outs[0], outs[1]) < 1e-12


def test_dtn_identities_laplace():
    # Pin P5: for c = 0 the DtN map kills constants, and maps x to the flux pattern
    # (0 on S/N, 1 on E/W) and y to (1 on S/N, 0 on E/W): exact for leaves and merges.
    p, q = 10, 9
    t = tr.uniform_tree(0, 0, 1, 1, 2, 2, q)
    X, Y = leaf_points(t, p)
    coeffs, _ = syn.poisson_manufactured(X, Y)
    ops = hps.build(t, np.array(coeffs), p)
    gp = t.gauss_points()
    for bid, b in enumerate(t.boxes):
        T = ops[bid]["T"]
        xs, ys = gp[b.ge, 0], gp[b.ge, 1]
        assert np.max(np.abs(T @ np.ones(len(b.ge)))) < 1e-10 * np.max(np.abs(T))
        vx, vy = T @ xs, T @ ys
        x0, y0, x1, y1 = b.rect
        on_vert = (np.isclose(xs, x0) | np.isclose(xs, x1))
        assert np.allclose(vx, np.where(on_vert, 1.0, 0.0), atol=1e-9)
        assert np.allclose(vy, np.where(on_vert, 0.0, 1.0), atol=1e-9)


def test_dtn_symmetry_self_adjoint():
    # Pin P5b: for A = -c11 d_xx - c22 d_yy + c (constants), u = exp(a x + b y) with
    # c11 a^2 + c22 b^2 = c solves A u = 0.  T must map its Gauss trace to its exact
    # fluxes (a u on E/W, b u on S/N), and the Green identity
    # sum_W (u sigma K T v - v sigma K T u) = 0 (outward signs sigma, conormal factor K =
    # c22 on S/N and c11 on E/W, Gauss weights W) must hold; both errors decay with p.
    c11, c22, c0 = 1.0, 1.5, 2.0
    sols = []
    for a in (0.7, -1.1):
        b = np.sqrt((c0 - c11 * a * a) / c22)
        sols.append((a, b))
    flux_err, green = [], []
    for p in (8, 12, 16):
        q = p - 1
        h = 0.5
        n2 = p * p
        coeffs = [np.full(n2, c11), np.zeros(n2), np.full(n2, c22), np.zeros(n2), np.zeros(n2), np.full(n2, c0)]
        T = lfm.leaf_ops(coeffs, p, q, h, h)["T"]
        gx, gy = sp.leaf_gauss_points(0.0, 0.0, h, h, q)
        _, w = sp.gauss_nodes(q)
        sig = np.concatenate([-c22 * np.ones(q), c11 * np.ones(q), c22 * np.ones(q), -c11 * np.ones(q)])
        W = np.tile(w * h / 2, 4) * sig
        tr_ = [np.exp(a * gx + b * gy) for a, b in sols]
        err = 0.0
        for (a, b), u in zip(sols, tr_):
            exact = np.concatenate([b * u[:q], a * u[q:2 * q], b * u[2 * q:3 * q], a * u[3 * q:]])
            err = max(err, np.max(np.abs(T @ u - exact)) / np.max(np.abs(exact)))
        flux_err.append(err)
        u, v = tr_
        green.append(abs(np.dot(u, W * (T @ v)) - np.dot(v, W * (T @ u))))
    assert flux_err[-1] < 1e-10 and flux_err[-1] < 1e-3 * flux_err[0]
    assert green[-1] < 1e-10


def test_flux_continuity_and_residual():
    # Pin P6: after a solve the leaf fluxes from both sides of every interior edge agree,
    # i.e. every equation of the global system has a rounding-level residual.
    p = 9
    t = tr.uniform_tree(0, 0, 1, 1, 3, 2, p - 1)
    coeffs, g, f, _ = _problem(t, p)
    ops = hps.build(t, coeffs, p)
    uc, ug = hps.solve(t, ops, p, f, g)
    r_ci, r_jump, r_bdry = hps.residual(t, coeffs, p, f, g, uc, ug)
    v = hps.leaf_fluxes(t, p, uc)
    assert np.max(np.abs(r_jump)) < 1e-10 * np.max(np.abs(v))
    assert np.max(np.abs(r_ci)) < 1e-10 * np.max(np.abs(g))
    assert np.max(np.abs(r_bdry)) == 0.0


def test_correction_solve_with_jump_residual():
    # The residual (r_ci, r_jump) of a perturbed iterate, fed back as a load and a flux-jump
    # right-hand side, gives the exact correction in one solve.
    p = 8
    t = tr.uniform_tree(0, 0, 1, 1, 2, 2, p - 1)
    coeffs, g, f, _ = _problem(t, p)
    ops = hps.build(t, coeffs, p)
    uc, ug = hps.solve(t, ops, p, f, g)
    rng = np.random.default_rng(5)
    ug2 = ug + 1e-3 * rng.standard_normal(ug.shape)
    ug2[t.boundary] = ug[t.boundary]
    uc2 = uc + 1e-3 * rng.standard_normal(uc.shape)
    r_ci, r_jump, _ = hps.residual(t, coeffs, p, f, g, uc2, ug2)
    _, ci, _ = sp.leaf_index_sets(p)
    gcorr = np.zeros_like(uc)
    gcorr[:, ci] = r_ci
    dc, dg = hps.solve(t, ops, p, np.zeros((len(t.boundary), 1)), gcorr, r_jump)
    ce, _, _ = sp.leaf_index_sets(p)
    fixed = uc2 + dc
    L = sp.L_ce_ge(p, t.q)
    for lf in range(t.n_leaves):
        fixed[lf][ce] = L @ (ug2 + dg)[t.boxes[t.leaves[lf]].ge]
    assert rel_linf(fixed, uc) < 1e-10
    assert rel_linf(ug2 + dg, ug) < 1e-10


def test_single_leaf_equals_direct_collocation():
    # Pin P7: a 1 x 1 tree is the plain Chebyshev collocation solve with Dirichlet rows
    # u_ce = L_ce,ge f.
    p = 11
    t = tr.uniform_tree(0, 0, 0.5, 0.5, 1, 1, p - 1)
    coeffs, g, f, _ = _problem(t, p)
    uc, _ = hps.solve(t, hps.build(t, coeffs, p), p, f, g)
    A = lfm.leaf_A([coeffs[k][0] for k in range(6)], p, 0.5, 0.5)
    ce, ci, _ = sp.leaf_index_sets(p)
    M = A.copy()
    rhs = g[0].copy()
    M[ce] = 0.0
    M[ce, ce] = 1.0
    rhs[ce] = sp.L_ce_ge(p, p - 1) @ f
    assert rel_linf(uc[0, :, 0], np.linalg.solve(M, rhs)) < 1e-11


def test_heat_eigenmode_backward_euler():
    # Pin P12: (I - dt Laplace) u^{n+1} = u^n, u^0 = sin(pi x) sin(pi y), f = 0 gives
    # u^n = (1 + 2 pi^2 dt)^{-n} u^0 up to the (spectrally small) spatial error.
    p, dt, nsteps = 14, 1e-3, 5
    t = tr.uniform_tree(0, 0, 1, 1, 2, 2, p - 1)
    X, Y = leaf_points(t, p)
    n2 = p * p
    coeffs = np.array([np.full((t.n_leaves, n2), dt), np.zeros((t.n_leaves, n2)), np.full((t.n_leaves, n2), dt),
                       np.zeros((t.n_leaves, n2)), np.zeros((t.n_leaves, n2)), np.ones((t.n_leaves, n2))])
    ops = hps.build(t, coeffs, p)
    u = np.sin(np.pi * X) * np.sin(np.pi * Y)
    u0 = u.copy()
    f = np.zeros(len(t.boundary))
    for _ in range(nsteps):
        u = hps.solve(t, ops, p, f, u)[0][..., 0]
    expect = (1 + 2 * np.pi ** 2 * dt) ** (-nsteps) * u0
    assert np.max(np.abs(u - expect)) < 1e-9
