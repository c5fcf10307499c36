"""Brute force: the global collocation system that Algorithms 1-2 eliminate, assembled
densely and solved with numpy.linalg.solve (tiny meshes only).

Unknowns z = [u_g (all Gaussian nodes) ; u_ci of leaf 0 ; u_ci of leaf 1 ; ...].
Equations, in this order:
  1. every leaf interior Chebyshev node i:  A_ci,ci u_ci + A_ci,ce L_ce,ge u_ge = g_ci
     (Eqs. local_sol and alpine2p5),
  2. every Gaussian node j on an interface, one equation each:
     - shared by the W/S leaf a and the E/N leaf b:
       (D_ge,c u_c)_a(j) - (D_ge,c u_c)_b(j) = rho_j   (flux continuity, Sec. 4 / Eq. pair);
     - a fine node on a coarsened side of a refined parent (Sec. 6.4):
       u_j - (P_up u_coarse)_j = 0;
     - a coarse node facing a refined parent: the coarse leaf's flux minus the P_down
       projection of the fine leaves' fluxes (W/S side minus E/N side) = rho_j,
  3. every boundary Gaussian node: u_j = f_j   (Eq. basic, Algorithm 2 root step); with
     other boundary kinds (Sec. 7.6, ``oracle.boundary``): for each periodic west node j
     and its east partner e, u_j - u_e = 0 and (D_ge,c u_c)_east leaf(e) -
     (D_ge,c u_c)_west leaf(j) = 0 (flux continuity across the seam); on a Neumann side
     (D_ge,c u_c)(j) = f_j,
with u_c = [L_ce,ge u_ge on I_ce ; u_ci on I_ci] on each leaf.

This module is oracle code (test infrastructure); see ``oracle/__init__.py``.
"""
import numpy as np

from . import boundary as bd
from . import spectral as sp
from .leaf import leaf_A

# A node on a leaf's E or N side lies on the W/S side of the interface it belongs to.
SIDES_WS = {0: False, 1: True, 2: True, 3: False}


def _boundary_rows(tree, bc):
    """Boundary equations in order: ("dir", j), ("neu", j) or ("seam", j, e)."""
    we, sn = (bd.DIRICHLET, bd.DIRICHLET) if bc is None else bc
    partner = {}
    if we == bd.PERIODIC:
        W, E = bd.periodic_pairs(tree)
        partner = {int(w): int(e) for w, e in zip(W, E)}
        east = set(int(e) for e in E)
    else:
        east = set()
    neu = set()
    if sn == bd.NEUMANN:
        _, _, S, N = bd.classify(tree)
        neu = set(int(g) for g in S) | set(int(g) for g in N)
    rows = []
    for j in tree.boundary:
        j = int(j)
        if j in partner:
            rows.append(("seam", j, partner[j]))
        elif j in east:
            continue
        elif j in neu:
            rows.append(("neu", j))
        else:
            rows.append(("dir", j))
    return rows


def assemble(tree, coeffs, p, bc=None):
    """Return (K, meta): the dense system matrix and the index bookkeeping."""
    q = tree.q
    ce, ci, _ = sp.leaf_index_sets(p)
    m = len(ci)
    L = sp.L_ce_ge(p, q)
    ng = tree.n_gauss
    nl = tree.n_leaves
    n = ng + nl * m
    K = np.zeros((n, n))
    row = 0
    # map from leaf-local u_c (p^2) to global unknowns: u_c = E_l z
    E = []
    for lf in range(nl):
        b = tree.boxes[tree.leaves[lf]]
        El = np.zeros((p * p, n))
        El[np.ix_(ce, b.ge)] = L
        El[ci, ng + lf * m + np.arange(m)] = 1.0
        E.append(El)
    Arows = []
    for lf in range(nl):
        x0, y0, x1, y1 = tree.leaf_rect(lf)
        A = leaf_A([coeffs[k][lf] for k in range(6)], p, x1 - x0, y1 - y0)
        K[row:row + m] = A[ci] @ E[lf]
        Arows.append(A[ci])
        row += m
    flux = []
    for lf in range(nl):
        x0, y0, x1, y1 = tree.leaf_rect(lf)
        flux.append(sp.D_ge_c(p, q, x1 - x0, y1 - y0) @ E[lf])
    for la, pa, lb, pb in tree.interior_pairs:
        K[row] = flux[la][pa] - flux[lb][pb]
        row += 1
    # coarse-fine interfaces of refined parents
    own = tree.owners
    for g in sorted(tree.slave):
        bid, r = tree.slave[g]
        b = tree.boxes[bid]
        K[row, g] = 1.0
        K[row, b.ge] -= b.Pup[r]
        row += 1
    for g in sorted(tree.coarse_of):
        bid, r = tree.coarse_of[g]
        b = tree.boxes[bid]
        (lc, pc), = own[g]
        proj = np.zeros(n)
        for k, gf in enumerate(b.ge_old):
            if b.Pdown[r, k] != 0.0 and gf in tree.slave:
                (lf, pf), = own[gf]
                proj += b.Pdown[r, k] * flux[lf][pf]
        coarse_is_ws = SIDES_WS[pc // q]
        K[row] = (flux[lc][pc] - proj) if coarse_is_ws else (proj - flux[lc][pc])
        row += 1
    for r in _boundary_rows(tree, bc):
        if r[0] == "dir":
            K[row, r[1]] = 1.0
            row += 1
        elif r[0] == "neu":
            (lb, pb), = own[r[1]]
            K[row] = flux[lb][pb]
            row += 1
        else:
            j, e = r[1], r[2]
            K[row, j] = 1.0
            K[row, e] = -1.0
            (lw, pw), = own[j]
            (le, pe), = own[e]
            K[row + 1] = flux[le][pe] - flux[lw][pw]
            row += 2
    assert row == n, "every Gaussian node needs exactly one interface or boundary equation"
    return K, {"E": E, "m": m, "ci": ci, "ng": ng}


def rhs(tree, p, f, g, rho=None, bc=None):
    """Right-hand side of the assembled system, same equation order."""
    _, ci, _ = sp.leaf_index_sets(p)
    g = np.asarray(g, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    if g.ndim == 2:
        g = g[..., None]
    if f.ndim == 1:
        f = f[:, None]
    nrhs = g.shape[-1]
    parts = [g[lf][ci] for lf in range(tree.n_leaves)]
    if rho is None:
        parts.append(np.zeros((len(tree.interior_pairs), nrhs)))
    else:
        rho = np.asarray(rho, dtype=np.float64).reshape(tree.n_gauss, -1)
        parts.append(rho[tree.interior])
    parts.append(np.zeros((len(tree.slave), nrhs)))
    if rho is None:
        parts.append(np.zeros((len(tree.coarse_of), nrhs)))
    else:
        parts.append(rho[sorted(tree.coarse_of)])
    brow = {int(j): k for k, j in enumerate(tree.boundary)}
    fb = []
    for r in _boundary_rows(tree, bc):
        if r[0] == "seam":
            fb += [np.zeros(nrhs), np.zeros(nrhs)]
        else:
            fb.append(f[brow[r[1]]])
    parts.append(np.array(fb).reshape(-1, nrhs))
    return np.vstack(parts)


def solve(tree, coeffs, p, f, g, rho=None, bc=None):
    """Dense solve; returns (u_c (n_leaf, p^2, nrhs), u_g (n_gauss, nrhs))."""
    K, meta = assemble(tree, coeffs, p, bc)
    b = rhs(tree, p, f, g, rho, bc)
    if bc is None or tuple(bc) == (bd.DIRICHLET, bd.DIRICHLET):
        z = np.linalg.solve(K, b)
    else:
        # without Dirichlet data on some side the Gaussian unknowns can carry directions
        # that no Chebyshev value sees (``oracle.boundary``): least squares picks one
        z = np.linalg.lstsq(K, b, rcond=1e-10)[0]
    u_c = np.array([El @ z for El in meta["E"]])
    return u_c, z[:meta["ng"]]


def solve_transpose(tree, coeffs, p, ubar):
    """The adjoint by brute force: lambda = K^-T (dJ/dz), with dJ/dz = sum_l E_l^T ubar_l.
    Returns (fbar, gbar, rhobar) laid out like oracle.hps.adjoint."""
    K, meta = assemble(tree, coeffs, p)
    ubar = np.asarray(ubar, dtype=np.float64)
    if ubar.ndim == 2:
        ubar = ubar[..., None]
    dz = sum(meta["E"][lf].T @ ubar[lf] for lf in range(tree.n_leaves))
    lam = np.linalg.solve(K.T, dz)
    m, ci = meta["m"], meta["ci"]
    nl = tree.n_leaves
    gbar = np.zeros((nl, p * p, ubar.shape[-1]))
    for lf in range(nl):
        gbar[lf][ci] = lam[lf * m:(lf + 1) * m]
    nint = len(tree.interior_pairs)
    rhobar = np.zeros((tree.n_gauss, ubar.shape[-1]))
    rhobar[tree.interior] = lam[nl * m:nl * m + nint]
    nsl, nco = len(tree.slave), len(tree.coarse_of)
    off = nl * m + nint + nsl
    rhobar[sorted(tree.coarse_of)] = lam[off:off + nco]
    fbar = lam[off + nco:]
    return fbar, gbar, rhobar
