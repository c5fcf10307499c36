"""Pins for the oracle's reference-element operators (Sec. 3.1-3.4) against closed forms."""
import numpy as np
import pytest

from oracle import spectral as sp
from oracle import tree as tr


@pytest.mark.parametrize("p", [6, 9, 16, 20])
def test_diff_matrix_exact_on_polynomials(p):
    # Sec. 3.2: differentiation is exact for polynomials of degree <= p-1.
    x = sp.cheb_nodes(p)
    D = sp.diff_matrix(x)
    for k in range(p):
        du = D @ x ** k
        exact = k * x ** (k - 1) if k else np.zeros_like(x)
        assert np.max(np.abs(du - exact)) < 1e-12 * max(1, k * k) * p * p


def test_diff_matrix_matches_textbook_chebyshev_formula():
    # Independent closed form (Trefethen, Spectral Methods in MATLAB, cheb.m) on descending
    # nodes cos(pi j/N); reversing both axes gives the ascending-node matrix.
    p = 12
    N = p - 1
    xd = np.cos(np.pi * np.arange(p) / N)
    c = np.ones(p)
    c[0] = c[-1] = 2.0
    D = np.zeros((p, p))
    for i in range(p):
        for j in range(p):
            if i != j:
                D[i, j] = (c[i] / c[j]) * (-1.0) ** (i + j) / (xd[i] - xd[j])
    D[0, 0] = (2 * N * N + 1) / 6.0
    D[N, N] = -(2 * N * N + 1) / 6.0
    for i in range(1, N):
        D[i, i] = -xd[i] / (2 * (1 - xd[i] ** 2))
    Dasc = D[::-1, ::-1]
    assert np.max(np.abs(Dasc - sp.diff_matrix(sp.cheb_nodes(p)))) < 1e-11


@pytest.mark.parametrize("q", [5, 15, 19])
def test_gauss_legendre_quadrature(q):
    x, w = sp.gauss_nodes(q)
    assert np.all(np.diff(x) > 0)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


@pytest.mark.parametrize("n", [5, 15])
def test_interp_exact_including_extrapolation(n):
    xs = sp.gauss_nodes(n)[0]
    t = np.array([-1.0, -0.7, 0.0, 0.3, 1.0])
    P = sp.interp_matrix(xs, t)
    for k in range(n):
        assert np.max(np.abs(P @ xs ** k - t ** k)) < 1e-12


@pytest.mark.parametrize("p", [6, 16])
def test_L_ce_ge_exact_for_polynomials_and_corners(p):
    # Eq. alpine2p5: side interpolation from q Gauss nodes; corners are the mean of the two
    # extrapolations, which both equal the exact corner value for degree <= q-1 data.
    q = p - 1
    ce, _, _ = sp.leaf_index_sets(p)
    L = sp.L_ce_ge(p, q)
    assert L.shape == (4 * (p - 1), 4 * q)
    X, Y = sp.leaf_cheb_points(-1, -1, 2, 2, p)
    gx, gy = sp.leaf_gauss_points(-1, -1, 2, 2, q)
    for a, b in [(0, 0), (1, 0), (3, q - 1), (q - 1, q - 1)]:
        assert np.max(np.abs(L @ (gx ** a * gy ** b) - (X ** a * Y ** b)[ce])) < 1e-10
    # corner rows: exactly two non-zero blocks of weight one half
    k_sw = list(ce).index(0)
    assert abs(L[k_sw, :q].sum() - 0.5) < 1e-13 and abs(L[k_sw, 3 * q:].sum() - 0.5) < 1e-13
    assert np.all(L[k_sw, q:3 * q] == 0.0)


def test_D_ge_c_exact_fluxes():
    # Sec. 3.4: d/dy on S and N, d/dx on E and W, at the Gauss nodes.
    p, q = 10, 9
    x0, y0, hx, hy = 0.25, -0.5, 0.5, 0.75
    X, Y = sp.leaf_cheb_points(x0, y0, hx, hy, p)
    gx, gy = sp.leaf_gauss_points(x0, y0, hx, hy, q)
    Dg = sp.D_ge_c(p, q, hx, hy)
    a, b = 4, 7
    v = Dg @ (X ** a * Y ** b)
    ux = a * gx ** (a - 1) * gy ** b
    uy = b * gx ** a * gy ** (b - 1)
    exact = np.concatenate([uy[:q], ux[q:2 * q], uy[2 * q:3 * q], ux[3 * q:]])
    assert np.max(np.abs(v - exact)) < 1e-10 * np.max(np.abs(exact))


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_dof_formula_matches_unique_chebyshev_nodes():
    # Sec. 7: N = n^2 (p-1)^2 + 2 n (p-1) + 1 distinct Chebyshev nodes on an n x n grid.
    for n, p, N in ((int(a), int(b), int(c)) for a, b, c in _golden("dof_counts.txt")):
        if n > 4:
            continue  # counted only on small grids; the formula rows are checked below
        t = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
        pts = set()
        for lf in range(t.n_leaves):
            x0, y0, x1, y1 = t.leaf_rect(lf)
            X, Y = sp.leaf_cheb_points(x0, y0, x1 - x0, y1 - y0, p)
            pts.update(zip(np.round(X, 12), np.round(Y, 12)))
        assert len(pts) == N
    for n, p, N in ((int(a), int(b), int(c)) for a, b, c in _golden("dof_counts.txt")):
        assert n * n * (p - 1) ** 2 + 2 * n * (p - 1) + 1 == N


def test_refinement_count_matches_paper():
    # Sec. 7.3: 4 x 4 leaves plus one level of refinement gives 28 leaf boxes.
    for row in _golden("refinement_counts.txt"):
        n, lev, xh, yh, cnt = int(row[0]), int(row[1]), float(row[2]), float(row[3]), int(row[4])
        rects = [(i / n, j / n, (i + 1) / n, (j + 1) / n) for j in range(n) for i in range(n)]
        assert len(tr.refine_rects(rects, (xh, yh), lev)) == cnt
