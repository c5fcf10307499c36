"""Leaf computation (Sec. 3; Algorithm 1, leaf branch).

Coefficient arrays are the six fields of Eq. defA tabulated at the p^2 Chebyshev nodes of
the leaf (node index iy * p + ix), in the order c11, c12, c22, c1, c2, c.

This module is oracle code (test infrastructure); see ``oracle/__init__.py``.
"""
import numpy as np

from . import spectral as sp

COEFF_NAMES = ("c11", "c12", "c22", "c1", "c2", "c")


def leaf_A(coeffs, p, hx, hy):
    """The p^2 x p^2 collocation matrix of Sec. 3.2,
    A = -C11 D1^2 - 2 C12 D1 D2 - C22 D2^2 + C1 D1 + C2 D2 + C,
    with the C's diagonal matrices of nodal coefficient values."""
    c11, c12, c22, c1, c2, c0 = [np.asarray(c, dtype=np.float64) for c in coeffs]
    D1, D2 = sp.diff_ops(p, hx, hy)
    A = (-c11[:, None] * (D1 @ D1)
         - 2.0 * c12[:, None] * (D1 @ D2)
         - c22[:, None] * (D2 @ D2)
         + c1[:, None] * D1
         + c2[:, None] * D2
         + np.diag(c0))
    return A


def leaf_ops(coeffs, p, q, hx, hy):
    """All operators of one leaf, written exactly as Algorithm 1 (leaf branch) states them.

    Returns a dict with
      F : p^2 x m,  F_c,ci = [0 ; A_ci,ci^-1]                       (Eq. alpine1)
      S : p^2 x 4q, S_c,ge = [I ; -A_ci,ci^-1 A_ci,ce] L_ce,ge          (Eqs. alpine2, alpine3)
      H : 4q x m,   H_ge,ci = D_ge,c F_c,ci                            (Eq. alpine4)
      T : 4q x 4q,  T_ge,ge = D_ge,c S_c,ge                            (Eq. alpine4)
      A : the full collocation matrix; Dgec : D_ge,c; ce, ci : index sets.
    Rows of F and S are placed at their tensor node index (exterior rows of F are zero and
    exterior rows of S equal L_ce,ge).
    """
    A = leaf_A(coeffs, p, hx, hy)
    ce, ci, _ = sp.leaf_index_sets(p)
    Acici = A[np.ix_(ci, ci)]
    Acice = A[np.ix_(ci, ce)]
    L = sp.L_ce_ge(p, q)
    Ainv = np.linalg.inv(Acici)
    n2, m = p * p, len(ci)
    F = np.zeros((n2, m))
    F[ci, :] = Ainv
    S = np.zeros((n2, 4 * q))
    S[ce, :] = L
    S[ci, :] = -Ainv @ Acice @ L
    Dgec = sp.D_ge_c(p, q, hx, hy)
    H = Dgec @ F
    T = Dgec @ S
    return {"F": F, "S": S, "H": H, "T": T, "A": A, "Dgec": Dgec, "ce": ce, "ci": ci, "L": L}


def apply_A(coeffs, u, p, hx, hy):
    """(A u) at all p^2 nodes for nodal values u (p^2 or p^2 x nrhs), from the dense A."""
    return leaf_A(coeffs, p, hx, hy) @ u
