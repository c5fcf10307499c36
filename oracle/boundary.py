"""Root boundary conditions other than Dirichlet data, for the parabolic example of
Sec. 7.6: periodic west/east sides and flux (Neumann) data on the south/north sides.

At the root, Algorithm 2's upward pass ends with the DtN relation of the whole domain
(Sec. 4 applied to the root box): on the boundary Gaussian nodes, v = T u + h, with v the
flux (the paper's sign convention, Sec. 2: d/dx on vertical sides, d/dy on horizontal
ones, not the outward normal derivative).

Periodic west/east sides identify each west node with the east node at the same height,
u_W = u_E = u_s, and ask for equal fluxes v_E = v_W.  Writing the remaining boundary
nodes as x:
    v_E - v_W = (T_EE + T_EW - T_WE - T_WW) u_s + (T_Ex - T_Wx) u_x + h_E - h_W = 0,
so u_s = X_s (R_s u_x + d_s) with X_s = Z_s^-1, Z_s = (T_EE + T_EW) - (T_WE + T_WW),
R_s = T_Wx - T_Ex, d_s = h_W - h_E: the merge of Sec. 4 with the root glued to itself.
The flux on the remaining nodes is then v_x = T' u_x + h' with
    T' = T_xx + C_s X_s R_s,  h' = h_x + C_s X_s d_s,  C_s = T_xE + T_xW.
Flux data on a set N of the remaining nodes (the rest, D, keep Dirichlet data) give
    u_N = T'_NN^-1 (f_N - h'_N - T'_ND u_D).
Then u_s = X_s (R_s u_x + d_s) and the downward pass of Algorithm 2 runs unchanged.

When no side carries Dirichlet data the flux system T'_NN can be singular: the Gaussian-
node unknowns admit values that the corner-averaged interpolation L_ce,ge (Sec. 3.3) maps
to zero on every leaf (on a side, the polynomial of degree q - 1 that vanishes at the side's
p - 2 interior Chebyshev points, with the corner averages cancelling).  No Chebyshev value,
residual or flux sees such a direction, so T' maps it to zero and any solution of the flux
system gives the same u_c.  The oracle takes the least-squares solution with singular
values below 1e-9 of the largest treated as zero.

This module is oracle code (test infrastructure); see ``oracle/__init__.py``.
"""
import numpy as np

DIRICHLET, PERIODIC, NEUMANN = "dirichlet", "periodic", "neumann"


def classify(tree):
    """Boundary Gaussian node ids by side: (W, E, S, N), W and E ordered by height (so
    W[k] and E[k] face each other), S and N by x."""
    gp = tree.gauss_points()
    x0, y0, x1, y1 = tree.boxes[0].rect
    b = np.asarray(tree.boundary)
    xs, ys = gp[b, 0], gp[b, 1]
    tol = 1e-12 * max(x1 - x0, y1 - y0)
    W = b[np.abs(xs - x0) < tol]
    E = b[np.abs(xs - x1) < tol]
    S = b[np.abs(ys - y0) < tol]
    N = b[np.abs(ys - y1) < tol]
    W = W[np.argsort(gp[W, 1], kind="stable")]
    E = E[np.argsort(gp[E, 1], kind="stable")]
    S = S[np.argsort(gp[S, 0], kind="stable")]
    N = N[np.argsort(gp[N, 0], kind="stable")]
    if len(W) + len(E) + len(S) + len(N) != len(b):
        raise ValueError("boundary conditions by side need a rectangular domain")
    return W, E, S, N


def periodic_pairs(tree):
    """(W, E) with W[k] and E[k] at the same height; raises if the sides do not match."""
    W, E, _, _ = classify(tree)
    gp = tree.gauss_points()
    if len(W) != len(E) or np.max(np.abs(gp[W, 1] - gp[E, 1]), initial=0.0) > 1e-12:
        raise ValueError("periodic west/east sides need matching nodes")
    return W, E


def root_values(tree, T, h, f, bc):
    """Boundary values u at the root's exterior nodes (in ``tree.boxes[0].ge`` order) from
    the root DtN map T, its particular flux h (both in that order) and the boundary data
    f (rows in ``tree.boundary`` order: Dirichlet values, or flux values on Neumann sides;
    ignored on periodic sides).  bc = (west/east, south/north) kinds."""
    we, sn = bc
    ge = list(tree.boxes[0].ge)
    pos = {g: k for k, g in enumerate(ge)}
    brow = {g: k for k, g in enumerate(tree.boundary)}
    W, E, S, N = classify(tree)
    u = np.zeros((len(ge), f.shape[1]))
    if we == PERIODIC:
        W, E = periodic_pairs(tree)
        xs = [g for g in ge if g not in set(W) | set(E)]
        iW, iE, ix = [pos[g] for g in W], [pos[g] for g in E], [pos[g] for g in xs]
        Z = (T[np.ix_(iE, iE)] + T[np.ix_(iE, iW)]) - (T[np.ix_(iW, iE)] + T[np.ix_(iW, iW)])
        R = T[np.ix_(iW, ix)] - T[np.ix_(iE, ix)]
        Cs = T[np.ix_(ix, iE)] + T[np.ix_(ix, iW)]
        Xs = np.linalg.inv(Z)
        ds = h[iW] - h[iE]
        Tp = T[np.ix_(ix, ix)] + Cs @ Xs @ R
        hp = h[ix] + Cs @ Xs @ ds
    else:
        xs = ge
        Tp, hp = T, h
    neu = set(S) | set(N) if sn == NEUMANN else set()
    kN = [k for k, g in enumerate(xs) if g in neu]
    kD = [k for k, g in enumerate(xs) if g not in neu]
    ux = np.zeros((len(xs), f.shape[1]))
    for k in kD:
        ux[k] = f[brow[xs[k]]]
    if kN:
        fN = np.array([f[brow[xs[k]]] for k in kN])
        rhs = fN - hp[kN] - Tp[np.ix_(kN, kD)] @ ux[kD]
        ux[kN] = np.linalg.lstsq(Tp[np.ix_(kN, kN)], rhs, rcond=1e-9)[0]
    for k, g in enumerate(xs):
        u[pos[g]] = ux[k]
    if we == PERIODIC:
        us = Xs @ (R @ ux + ds)
        u[iW] = us
        u[iE] = us
    return u
