"""The identity behind the blocked merge elimination, checked on the CPU with a plain
in-place Gauss-Jordan elimination written here (not the library's code).

A merge matrix M = [[Z, R], [B, T]] (Algorithm 1: Z the interface block, pivots chosen by
partial pivoting among its K rows only, rows never swapped physically) is eliminated in
place over its first K columns.  Every pivot row comes from the top block, so each bottom
row x = [x_L | x_R] ends as [0 | x_R] - x_L Top, Top[k] being the final state of the pivot
row of column k.  The blocked form eliminates the top rows alone and then forms the bottom
rows with that one product; both must give the same matrix to rounding.
"""
import numpy as np
import pytest


def gj_in_place(M, K, rows):
    """Gauss-Jordan elimination of columns 0 .. K-1 of M in place, pivots chosen among the
    top K rows (largest magnitude, the first among equals), applied to rows [0, rows).
    Returns the logical-to-physical pivot map."""
    perm = list(range(K))
    for j in range(K):
        cand = perm[j:]
        r = max(cand, key=lambda i: (abs(M[i, j]), -i))
        k = perm.index(r)
        perm[j], perm[k] = perm[k], perm[j]
        p = perm[j]
        piv = M[p, j]
        prow = M[p, :].copy()
        for i in range(rows):
            if i == p:
                continue
            f = M[i, j] / piv
            M[i, :] -= f * prow
            M[i, j] = -f
        M[p, :] = prow / piv
        M[p, j] = 1.0 / piv
    return perm


@pytest.mark.parametrize("K,k12,seed", [(6, 10, 0), (16, 40, 1), (33, 70, 2)])
def test_bottom_rows_are_one_product_with_the_eliminated_top_rows(K, k12, seed):
    rng = np.random.default_rng(seed)
    R = K + k12
    M = rng.standard_normal((R, R))
    M[:K, :K] += 3.0 * np.eye(K)          # a well-conditioned interface block
    full = M.copy()
    gj_in_place(full, K, R)                # the panel form: every row updated
    top = M.copy()
    perm = gj_in_place(top, K, K)          # the blocked form: top rows only ...
    T0 = M[K:, :].copy()
    BL = T0[:, :K].copy()
    base = T0.copy()
    base[:, :K] = 0.0
    Top = top[perm, :]                     # pivot rows in pivot (column) order
    bottom = base - BL @ Top               # ... then one product
    scale = np.max(np.abs(full))
    assert np.max(np.abs(top[:K] - full[:K])) <= 1e-12 * scale
    assert np.max(np.abs(bottom - full[K:])) <= 1e-12 * scale


def test_identity_reproduces_the_schur_complement():
    # the bottom-right block is T - B Z^-1 R whatever the pivot order, and the bottom-left
    # block -B Z^-1 with its columns in pivot order (column j belongs to physical row
    # perm[j]: the extraction un-permutes them)
    rng = np.random.default_rng(5)
    K, k12 = 12, 20
    M = rng.standard_normal((K + k12, K + k12))
    M[:K, :K] += 2.0 * np.eye(K)
    Z, Rb, B, T = M[:K, :K], M[:K, K:], M[K:, :K], M[K:, K:]
    full = M.copy()
    perm = gj_in_place(full, K, K + k12)
    Zi = np.linalg.inv(Z)
    assert perm != list(range(K))          # the case exercises pivoting
    assert np.allclose(full[K:, K:], T - B @ Zi @ Rb, rtol=0, atol=1e-11)
    assert np.allclose(full[K:, :K], (-B @ Zi)[:, perm], rtol=0, atol=1e-11)
