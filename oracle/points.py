"""Node coordinates of a tree for building inputs (test infrastructure, like the rest of
this package): the leaf Chebyshev nodes (Sec. 3.1) and the domain-boundary Gaussian
nodes (Sec. 2), computed from this package's own tables."""
import numpy as np

from . import spectral as sp


def leaf_points(tree, p):
    """(X, Y), each (n_leaf, p^2): leaf Chebyshev node coordinates, node iy * p + ix."""
    X, Y = [], []
    for lf in range(tree.n_leaves):
        x0, y0, x1, y1 = tree.leaf_rect(lf)
        x, y = sp.leaf_cheb_points(x0, y0, x1 - x0, y1 - y0, p)
        X.append(x)
        Y.append(y)
    return np.array(X), np.array(Y)


def boundary_points(tree):
    """(x, y) of the domain-boundary Gaussian nodes in boundary order (ascending id)."""
    gp = tree.gauss_points()
    return gp[tree.boundary, 0], gp[tree.boundary, 1]
