"""Pins of the oracle's periodic / Neumann root conditions (Sec. 7.6): the HPS solve with
the root DtN relation equals the dense global collocation system with seam and flux
equations, reproduces closed-form periodic-channel solutions, and Crank-Nicolson steps
of a Fourier mode follow the exact amplification factor."""
import numpy as np
import pytest

import synthetic as syn
from oracle import boundary as bd, dense, hps, leaf as lfm, tree as tr
from tests.helpers import boundary_points, leaf_points

BCS = [(bd.PERIODIC, bd.NEUMANN), (bd.PERIODIC, bd.DIRICHLET), (bd.DIRICHLET, bd.NEUMANN)]


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("nx,ny,p", [(1, 1, 7), (2, 2, 8), (4, 2, 7), (3, 2, 6)])
def test_root_conditions_match_dense_system(bc, nx, ny, p):
    t = tr.uniform_tree(0, 0, 1, 1, nx, ny, p - 1)
    X, Y = leaf_points(t, p)
    bx, by = boundary_points(t)
    prob = syn.VarCoeffProblem()
    coeffs = np.array(prob.coeffs(X, Y))
    coeffs[5] += 1.0     # keep the periodic / Neumann problem well away from singular
    g = np.stack([prob.load(X, Y), np.cos(2 * X) * Y], axis=-1)
    f = np.stack([np.sin(3 * bx) + by, bx * by], axis=-1)
    u, _ = hps.solve(t, hps.build(t, coeffs, p), p, f, g, bc=bc)
    ud, _ = dense.solve(t, coeffs, p, f, g, bc=bc)
    assert np.max(np.abs(u - ud)) < 1e-10 * np.max(np.abs(ud))


def _channel(eps=1 / 200, k=1e-2):
    """The Crank-Nicolson operator of Sec. 7.6, (I/k - A/2) with A = eps Laplace - d/dx:
    c11 = c22 = eps/2, c1 = 1/2, c = 1/k."""
    return eps, k


def test_periodic_channel_closed_form():
    # u = cos(2 pi x) cos(pi y): periodic in x, zero flux on y = 0, 1
    eps, k = _channel()
    n, p = 4, 16
    t = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(t, p)
    bx, _ = boundary_points(t)
    z = np.zeros_like(X)
    coeffs = np.array([z + eps / 2, z, z + eps / 2, z + 0.5, z, z + 1 / k])
    u = np.cos(2 * np.pi * X) * np.cos(np.pi * Y)
    ux = -2 * np.pi * np.sin(2 * np.pi * X) * np.cos(np.pi * Y)
    g = (eps / 2) * 5 * np.pi ** 2 * u + 0.5 * ux + u / k
    uh, _ = hps.solve(t, hps.build(t, coeffs, p), p, np.zeros_like(bx), g, bc=(bd.PERIODIC, bd.NEUMANN))
    assert np.max(np.abs(uh[..., 0] - u)) < 1e-9


def test_neumann_data_closed_form():
    # u = cos(2 pi x) sin(pi y) + x: flux d/dy = pi cos(2 pi x) cos(pi y) on S and N;
    # Dirichlet on W and E
    n, p = 3, 14
    t = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(t, p)
    bx, by = boundary_points(t)
    z = np.zeros_like(X)
    coeffs = np.array([z + 1, z, z + 1, z, z, z + 2])
    u = np.cos(2 * np.pi * X) * np.sin(np.pi * Y) + X
    g = 5 * np.pi ** 2 * np.cos(2 * np.pi * X) * np.sin(np.pi * Y) + 2 * u
    W, E, S, N = bd.classify(t)
    f = np.cos(2 * np.pi * bx) * np.sin(np.pi * by) + bx
    brow = {int(j): r for r, j in enumerate(t.boundary)}
    for j in list(S) + list(N):
        r = brow[int(j)]
        f[r] = np.pi * np.cos(2 * np.pi * bx[r]) * np.cos(np.pi * by[r])
    uh, _ = hps.solve(t, hps.build(t, coeffs, p), p, f, g, bc=(bd.DIRICHLET, bd.NEUMANN))
    assert np.max(np.abs(uh[..., 0] - u)) < 1e-9


def test_crank_nicolson_fourier_mode():
    # u0 = cos(2 pi x) cos(pi y); A e^{2 pi i x} cos(pi y) = lam (...) with
    # lam = -5 pi^2 eps - 2 pi i; CN multiplies the mode by (1/k + lam/2) / (1/k - lam/2)
    eps, k = _channel(k=2e-2)
    n, p, steps = 4, 16, 5
    t = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(t, p)
    bx, _ = boundary_points(t)
    z = np.zeros_like(X)
    M = np.array([z + eps / 2, z, z + eps / 2, z + 0.5, z, z + 1 / k])
    ops = hps.build(t, M, p)
    u = np.cos(2 * np.pi * X) * np.cos(np.pi * Y)
    for _ in range(steps):
        # right-hand side (I/k + A/2) u = (2/k) u - (I/k - A/2) u, applied per leaf
        Mu = np.array([lfm.apply_A(M[:, lf], u[lf], p, 1 / n, 1 / n) for lf in range(n * n)])
        u, _ = hps.solve(t, ops, p, np.zeros_like(bx), (2 / k) * u - Mu, bc=(bd.PERIODIC, bd.NEUMANN))
        u = u[..., 0]
    lam = -5 * np.pi ** 2 * eps - 2j * np.pi
    G = (1 / k + lam / 2) / (1 / k - lam / 2)
    exact = np.real(G ** steps * np.exp(2j * np.pi * X)) * np.cos(np.pi * Y)
    assert np.max(np.abs(u - exact)) < 1e-9


def test_null_directions_are_invisible_to_chebyshev_values():
    # periodic west/east + Neumann south/north with p = 8: the dense system is singular,
    # its null vector lives on the Gaussian unknowns only, every leaf's corner-averaged
    # interpolation L_ce,ge maps it to zero, and solutions differing by it give the same
    # u_c (the least-squares solution is taken)
    from oracle import spectral as sp
    p = 8
    t = tr.uniform_tree(0, 0, 1, 1, 2, 2, p - 1)
    X, Y = leaf_points(t, p)
    coeffs = np.array(syn.VarCoeffProblem().coeffs(X, Y))
    coeffs[5] += 1.0
    bc = (bd.PERIODIC, bd.NEUMANN)
    K, meta = dense.assemble(t, coeffs, p, bc)
    _, sv, Vt = np.linalg.svd(K)
    assert sv[-1] < 1e-11 * sv[0] < sv[-2]
    v = Vt[-1]
    ng = meta["ng"]
    assert np.max(np.abs(v[ng:])) < 1e-12
    L = sp.L_ce_ge(p, p - 1)
    for lf in range(t.n_leaves):
        assert np.max(np.abs(L @ v[t.boxes[t.leaves[lf]].ge])) < 1e-12
    g = np.cos(2 * X) * Y
    ud, _ = dense.solve(t, coeffs, p, np.zeros(len(t.boundary)), g, bc=bc)
    uh, _ = hps.solve(t, hps.build(t, coeffs, p), p, np.zeros(len(t.boundary)), g, bc=bc)
    assert np.max(np.abs(uh - ud)) < 1e-10 * np.max(np.abs(ud))
