"""Build and solve stages of the HPS solver (Algorithms 1 and 2), the FP64 residual of the
global collocation system, and the transposed sweeps (adjoint).

Array conventions (all FP64):
  coeffs : (6, n_leaf, p^2)      c11, c12, c22, c1, c2, c at every leaf Chebyshev node
  g      : (n_leaf, p^2, nrhs)   body load at the leaf Chebyshev nodes (interior ones used)
  f      : (n_bdry, nrhs)        Dirichlet data at the domain-boundary Gaussian nodes, in
                                 ascending global node id (``tree.boundary``)
  rho    : (n_gauss, nrhs)       optional right-hand side of the flux-continuity equations
                                 at interior Gaussian nodes (zero for Eq. basic)
  u_c    : (n_leaf, p^2, nrhs)   solution at the leaf Chebyshev nodes
  u_g    : (n_gauss, nrhs)       solution at the Gaussian nodes

This module is oracle code (test infrastructure); see ``oracle/__init__.py``.
"""
import numpy as np

from . import boundary as bd
from . import spectral as sp
from .leaf import leaf_ops, leaf_A


def _pos(lst):
    return {g: k for k, g in enumerate(lst)}


def build(tree, coeffs, p):
    """Algorithm 1: one upward sweep; leaf operators by Sec. 3, merges by Sec. 4.  A
    refined parent's DtN map is re-expressed on its coarsened sides, T_new = P_down T P_up
    (Sec. 6.3); its S keeps acting on the fine nodes, which the solve fills by P_up."""
    q = tree.q
    ops = {}
    for bid in tree.order_up():
        b = tree.boxes[bid]
        if b.children is None:
            x0, y0, x1, y1 = b.rect
            lf = b.leaf
            ops[bid] = leaf_ops([coeffs[k][lf] for k in range(6)], p, q, x1 - x0, y1 - y0)
            continue
        a, c = (tree.boxes[k] for k in b.children)
        Ta, Tb = ops[a.id]["T"], ops[c.id]["T"]
        pa, pb = _pos(a.ge), _pos(c.ge)
        I1 = [pa[g] for g in b.J1]
        I3a = [pa[g] for g in b.J3]
        I2 = [pb[g] for g in b.J2]
        I3b = [pb[g] for g in b.J3]
        T11, T13, T31, T33a = (Ta[np.ix_(r, s)] for r, s in ((I1, I1), (I1, I3a), (I3a, I1), (I3a, I3a)))
        T22, T23, T32, T33b = (Tb[np.ix_(r, s)] for r, s in ((I2, I2), (I2, I3b), (I3b, I2), (I3b, I3b)))
        X = np.linalg.inv(T33a - T33b)
        S = X @ np.hstack([-T31, T32])
        n1, n2 = len(I1), len(I2)
        Tblk = np.zeros((n1 + n2, n1 + n2))
        Tblk[:n1, :n1] = T11
        Tblk[n1:, n1:] = T22
        C = np.vstack([T13, T23])
        T = Tblk + C @ S
        if b.Pup is not None:
            T = b.Pdown @ T @ b.Pup
        ops[bid] = {"X": X, "S": S, "T": T, "C": C, "I1": I1, "I2": I2, "I3a": I3a, "I3b": I3b}
    return ops


def _as2d(a, lead):
    a = np.asarray(a, dtype=np.float64)
    return a.reshape(a.shape[:lead] + (-1,)) if a.ndim == lead else a


def solve(tree, ops, p, f, g, rho=None, bc=None):
    """Algorithm 2 (upward pass for particular solutions, downward pass for potentials),
    with per-box flux vectors h.  A non-zero ``rho`` enters the merge of the box whose J3
    holds the node: Eq. swiss with the continuity condition v3(alpha) - v3(beta) = rho3
    gives u3 = X (T32b u2 - T31a u1 + h3b - h3a + rho3).  Refined parents (Sec. 6.4): the
    upward flux is projected, h_new = P_down h_old, and on the way down the fine nodes of a
    coarsened side get u_fine = P_up u_coarse before the parent's S is applied.
    bc = (west/east, south/north) boundary kinds (``oracle.boundary``): with periodic or
    Neumann sides the root's boundary values come from the root DtN relation (Sec. 7.6),
    and f holds Dirichlet values or flux data per boundary node."""
    f = _as2d(f, 1)
    g = _as2d(g, 2)
    nrhs = g.shape[-1]
    _, ci, _ = sp.leaf_index_sets(p)
    if rho is not None:
        rho = _as2d(rho, 1)
    h, w = {}, {}
    for bid in tree.order_up():
        b = tree.boxes[bid]
        o = ops[bid]
        if b.children is None:
            h[bid] = o["H"] @ g[b.leaf][ci]
            continue
        a, c = b.children
        d = h[c][o["I3b"]] - h[a][o["I3a"]]
        if rho is not None:
            d = d + rho[b.J3]
        w[bid] = o["X"] @ d
        h[bid] = np.vstack([h[a][o["I1"]], h[c][o["I2"]]]) + o["C"] @ w[bid]
        if b.Pup is not None:
            h[bid] = b.Pdown @ h[bid]
    u_g = np.zeros((tree.n_gauss, nrhs))
    if bc is None or tuple(bc) == (bd.DIRICHLET, bd.DIRICHLET):
        u_g[tree.boundary] = f
    else:
        root = tree.boxes[0]
        u_g[root.ge] = bd.root_values(tree, ops[0]["T"], h[0], f, bc)
    u_c = np.zeros((tree.n_leaves, p * p, nrhs))
    for bid in range(len(tree.boxes)):
        b = tree.boxes[bid]
        o = ops[bid]
        if b.children is not None:
            if b.Pup is not None:
                fine = [k for k, g in enumerate(b.ge_old) if g not in set(b.ge)]
                u_g[np.array(b.ge_old)[fine]] = (b.Pup @ u_g[b.ge])[fine]
            u_g[b.J3] = o["S"] @ u_g[b.ge_old] + w[bid]
        else:
            u_c[b.leaf] = o["S"] @ u_g[b.ge] + o["F"] @ g[b.leaf][ci]
    return u_c, u_g


def leaf_fluxes(tree, p, u_c):
    """v_ge = D_ge,c u_c on every leaf (Sec. 3.4): (n_leaf, 4q, nrhs)."""
    out = []
    for lf in range(tree.n_leaves):
        x0, y0, x1, y1 = tree.leaf_rect(lf)
        out.append(sp.D_ge_c(p, tree.q, x1 - x0, y1 - y0) @ u_c[lf])
    return np.array(out)


def residual(tree, coeffs, p, f, g, u_c, u_g, rho=None):
    """Residual of the global collocation system solved by Algorithms 1-2:
      r_ci   = g_ci - A_ci,: u_c           at every leaf interior node (Eq. local_sol)
      r_jump = rho - (v_a - v_b)           at every interior Gaussian node, v = D_ge,c u_c
                                           from the W/S leaf a and the E/N leaf b
      r_bdry = f - u_g[boundary]
    where u_c on the exterior is rebuilt as L_ce,ge u_g (Eq. alpine2p5)."""
    g = _as2d(g, 2)
    q = tree.q
    ce, ci, _ = sp.leaf_index_sets(p)
    L = sp.L_ce_ge(p, q)
    uc = np.array(u_c, dtype=np.float64, copy=True)
    r_ci = np.zeros((tree.n_leaves, len(ci), uc.shape[-1]))
    for lf in range(tree.n_leaves):
        b = tree.boxes[tree.leaves[lf]]
        uc[lf][ce] = L @ u_g[b.ge]
        x0, y0, x1, y1 = b.rect
        A = leaf_A([coeffs[k][lf] for k in range(6)], p, x1 - x0, y1 - y0)
        r_ci[lf] = g[lf][ci] - A[ci] @ uc[lf]
    v = leaf_fluxes(tree, p, uc)
    pr = tree.interior_pairs
    r_jump = np.zeros((tree.n_gauss, uc.shape[-1]))
    jump = v[pr[:, 0], pr[:, 1]] - v[pr[:, 2], pr[:, 3]]
    if rho is not None:
        jump = _as2d(rho, 1)[tree.interior] - jump
    else:
        jump = -jump
    r_jump[tree.interior] = jump
    r_bdry = _as2d(f, 1) - u_g[tree.boundary]
    return r_ci, r_jump, r_bdry


def adjoint(tree, ops, p, ubar):
    """Transpose of the linear map (f, g, rho) -> u_c realised by Algorithm 2, applied to
    ubar = dJ/du_c: the downward pass transposed (leaves first, then parents from the
    bottom up), then the upward pass transposed (root first).  Returns (fbar, gbar, rhobar)
    with gbar zero at exterior Chebyshev nodes and rhobar zero off the interior nodes."""
    ubar = _as2d(ubar, 2)
    nrhs = ubar.shape[-1]
    _, ci, _ = sp.leaf_index_sets(p)
    ubar_g = np.zeros((tree.n_gauss, nrhs))
    gbar = np.zeros((tree.n_leaves, p * p, nrhs))
    wbar = {}
    for bid in tree.order_up():
        b = tree.boxes[bid]
        o = ops[bid]
        if b.children is None:
            ubar_g[b.ge] += o["S"].T @ ubar[b.leaf]
            gbar[b.leaf][ci] += o["F"].T @ ubar[b.leaf]
        else:
            wbar[bid] = ubar_g[b.J3].copy()
            ubar_g[b.ge_old] += o["S"].T @ ubar_g[b.J3]
            if b.Pup is not None:
                fine = [k for k, g in enumerate(b.ge_old) if g not in set(b.ge)]
                ubar_g[b.ge] += b.Pup[fine].T @ ubar_g[np.array(b.ge_old)[fine]]
    fbar = ubar_g[tree.boundary].copy()
    hbar = {bid: None for bid in range(len(tree.boxes))}
    rhobar = np.zeros((tree.n_gauss, nrhs))
    hbar[0] = np.zeros((len(tree.boxes[0].ge), nrhs))
    for bid in range(len(tree.boxes)):
        b = tree.boxes[bid]
        o = ops[bid]
        if b.children is None:
            gbar[b.leaf][ci] += o["H"].T @ hbar[bid]
            continue
        a, c = b.children
        n1 = len(o["I1"])
        if b.Pup is not None:
            hbar[bid] = b.Pdown.T @ hbar[bid]
        dbar = o["X"].T @ (wbar[bid] + o["C"].T @ hbar[bid])
        ha = np.zeros((len(tree.boxes[a].ge), nrhs))
        hc = np.zeros((len(tree.boxes[c].ge), nrhs))
        ha[o["I1"]] += hbar[bid][:n1]
        hc[o["I2"]] += hbar[bid][n1:]
        hc[o["I3b"]] += dbar
        ha[o["I3a"]] -= dbar
        hbar[a], hbar[c] = ha, hc
        rhobar[b.J3] = dbar
    return fbar, gbar, rhobar


def coeff_gradients(tree, p, u_c, gbar):
    """Gradients of a functional with respect to the nodal coefficients, from the adjoint
    load gbar (= the multipliers of the collocation equations) and the solution u_c.
    Row i of Eq. local_sol is (A u)_i = g_i with A from Sec. 3.2, so
    dJ/dc11 = gbar D1^2 u, dJ/dc12 = 2 gbar D1 D2 u, dJ/dc22 = gbar D2^2 u,
    dJ/dc1 = -gbar D1 u, dJ/dc2 = -gbar D2 u, dJ/dc = -gbar u  at interior nodes, 0 elsewhere.
    Returns (6, n_leaf, p^2), summed over right-hand sides."""
    u_c = _as2d(u_c, 2)
    gbar = _as2d(gbar, 2)
    _, ci, _ = sp.leaf_index_sets(p)
    out = np.zeros((6, tree.n_leaves, p * p))
    for lf in range(tree.n_leaves):
        x0, y0, x1, y1 = tree.leaf_rect(lf)
        D1, D2 = sp.diff_ops(p, x1 - x0, y1 - y0)
        u = u_c[lf]
        lam = gbar[lf]
        terms = (D1 @ D1 @ u, 2.0 * (D1 @ D2 @ u), D2 @ D2 @ u, -(D1 @ u), -(D2 @ u), -u)
        for k, t in enumerate(terms):
            out[k, lf, ci] = np.sum(lam[ci] * t[ci], axis=-1)
    return out
