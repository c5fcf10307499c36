"""Reference-element operators of the leaf discretisation (Sec. 3.1-3.4).

All matrices are for a leaf [x0, x0 + hx] x [y0, y0 + hy].  Node conventions:

* Chebyshev grid (Sec. 3.1): p Chebyshev-Lobatto points per direction, ascending;
  tensor node index ``k = iy * p + ix`` (x runs fastest).  The exterior set I_ce holds
  every node with ix or iy in {0, p-1} (4(p-1) nodes, corners included), the interior
  set I_ci the remaining (p-2)^2 nodes.  Both lists are in ascending node index.
* Gaussian boundary nodes (Sec. 3.1): q Gauss-Legendre points on each side, sides in
  the order S, E, N, W, each side ascending in its running coordinate (x on S/N, y on E/W).
* Fluxes (Sec. 3.1): d/dx on the vertical sides (E, W) and d/dy on the horizontal sides
  (S, N), never the outward normal derivative.

This module is oracle code (test infrastructure); see ``oracle/__init__.py``.
"""
import numpy as np

SIDES = ("S", "E", "N", "W")


def cheb_nodes(p):
    """Chebyshev-Lobatto points on [-1, 1], ascending (Sec. 3.1: a p x p Chebyshev grid
    whose exterior has 4(p-1) nodes, so the corners are grid points)."""
    k = np.arange(p)
    return -np.cos(np.pi * k / (p - 1))


def bary_weights(x):
    """Barycentric weights w_k = 1 / prod_{j != k} (x_k - x_j) (Berrut & Trefethen 2004, Eq. 3.2)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    w = np.empty(n)
    for k in range(n):
        d = x[k] - np.delete(x, k)
        w[k] = 1.0 / np.prod(d)
    return w


def interp_matrix(x_src, x_dst):
    """Lagrange interpolation matrix (len(x_dst) x len(x_src)) through the nodes x_src,
    in barycentric form (second form), exact for polynomials of degree < len(x_src).
    Targets outside the node range are extrapolations of the same polynomial."""
    x_src = np.asarray(x_src, dtype=np.float64)
    x_dst = np.asarray(x_dst, dtype=np.float64)
    w = bary_weights(x_src)
    P = np.zeros((len(x_dst), len(x_src)))
    for i, t in enumerate(x_dst):
        diff = t - x_src
        hit = np.nonzero(diff == 0.0)[0]
        if len(hit):
            P[i, hit[0]] = 1.0
            continue
        c = w / diff
        P[i] = c / c.sum()
    return P


def diff_matrix(x):
    """Spectral differentiation matrix on the nodes x (barycentric form, Berrut & Trefethen
    2004, Sec. 9): D_ij = (w_j / w_i) / (x_i - x_j) for i != j, and each diagonal entry is
    minus its row sum, so that D maps constants to zero.  Exact for polynomials of degree
    < len(x) (Sec. 3.2)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    w = bary_weights(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, np.arange(n) != i])
    return D


def gauss_nodes(q):
    """q Gauss-Legendre nodes on [-1, 1], ascending, and their weights (Sec. 2)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return x, w


def leaf_index_sets(p):
    """(I_ce, I_ci, side_nodes): exterior and interior node indices in ascending order, and
    for each side S, E, N, W the p node indices of that side in ascending running
    coordinate (the index sets I_s, I_e, I_n, I_w of Sec. 3.4)."""
    ce, ci = [], []
    for iy in range(p):
        for ix in range(p):
            k = iy * p + ix
            if ix in (0, p - 1) or iy in (0, p - 1):
                ce.append(k)
            else:
                ci.append(k)
    side = {
        "S": [0 * p + ix for ix in range(p)],
        "E": [iy * p + (p - 1) for iy in range(p)],
        "N": [(p - 1) * p + ix for ix in range(p)],
        "W": [iy * p + 0 for iy in range(p)],
    }
    return np.array(ce), np.array(ci), {s: np.array(v) for s, v in side.items()}


def L_loc(p, q):
    """q x p interpolation from the p Chebyshev points of one side to its q Gauss points
    (Sec. 3.4)."""
    return interp_matrix(cheb_nodes(p), gauss_nodes(q)[0])


def L_ce_ge(p, q):
    """The 4(p-1) x 4q matrix of Eq. alpine2p5.  Rows follow I_ce (ascending node index),
    columns the Gauss nodes S, E, N, W.  A non-corner exterior node takes the degree q-1
    interpolant of the Gauss data of its own side; a corner takes the mean of the two
    values extrapolated from the two sides that meet there (Sec. 3.4)."""
    ce, _, _ = leaf_index_sets(p)
    xc = cheb_nodes(p)
    xg = gauss_nodes(q)[0]
    G = interp_matrix(xg, xc)  # p x q: Gauss data of one side -> all p Chebyshev points of it
    L = np.zeros((len(ce), 4 * q))
    col = {s: slice(i * q, (i + 1) * q) for i, s in enumerate(SIDES)}
    for r, k in enumerate(ce):
        iy, ix = divmod(k, p)
        on = []
        if iy == 0:
            on.append(("S", ix))
        if ix == p - 1:
            on.append(("E", iy))
        if iy == p - 1:
            on.append(("N", ix))
        if ix == 0:
            on.append(("W", iy))
        wgt = 1.0 / len(on)
        for s, t in on:
            L[r, col[s]] += wgt * G[t]
    return L


def diff_ops(p, hx, hy):
    """Return (D1, D2): the p^2 x p^2 spectral differentiation matrices d/dx and d/dy on the
    Chebyshev grid of a leaf of size hx x hy (Sec. 3.2).  With x fastest, D1 = I (x) Dx and
    D2 = Dy (x) I."""
    D = diff_matrix(cheb_nodes(p))
    Dx = (2.0 / hx) * D
    Dy = (2.0 / hy) * D
    I = np.eye(p)
    return np.kron(I, Dx), np.kron(Dy, I)


def D_ge_c(p, q, hx, hy):
    """The 4q x p^2 flux matrix of Sec. 3.4: blocks L_loc D2(I_s,:), L_loc D1(I_e,:),
    L_loc D2(I_n,:), L_loc D1(I_w,:)."""
    D1, D2 = diff_ops(p, hx, hy)
    _, _, side = leaf_index_sets(p)
    Ll = L_loc(p, q)
    blocks = []
    for s in SIDES:
        Dsel = D2 if s in ("S", "N") else D1
        blocks.append(Ll @ Dsel[side[s], :])
    return np.vstack(blocks)


def leaf_cheb_points(x0, y0, hx, hy, p):
    """Coordinates (x, y) of the p^2 Chebyshev nodes of a leaf, node index iy * p + ix."""
    t = cheb_nodes(p)
    xs = x0 + 0.5 * hx * (t + 1.0)
    ys = y0 + 0.5 * hy * (t + 1.0)
    X, Y = np.meshgrid(xs, ys)  # X[iy, ix] = xs[ix]
    return X.ravel(), Y.ravel()


def leaf_gauss_points(x0, y0, hx, hy, q):
    """Coordinates of the 4q Gaussian boundary nodes of a leaf, order S, E, N, W."""
    g = gauss_nodes(q)[0]
    gx = x0 + 0.5 * hx * (g + 1.0)
    gy = y0 + 0.5 * hy * (g + 1.0)
    x = np.concatenate([gx, np.full(q, x0 + hx), gx, np.full(q, x0)])
    y = np.concatenate([np.full(q, y0), gy, np.full(q, y0 + hy), gy])
    return x, y
