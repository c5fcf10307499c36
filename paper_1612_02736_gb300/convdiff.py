"""Crank-Nicolson stepping of the convection-diffusion problem of Sec. 7.6 on a periodic
channel: u_t = eps Laplace(u) - du/dx on the unit square, periodic west/east sides and
zero flux on the south/north sides.

With A = eps Laplace - d/dx and step k, every step solves Eq. CN,
    (I/k - A/2) u^{n+1} = (I/k + A/2) u^n,
i.e. Eq. basic with c11 = c22 = eps/2, c1 = 1/2, c = 1/k (the operator is built once,
Algorithm 1) and the right-hand side (I/k + A/2) u^n = 2/k u^n - (I/k - A/2) u^n evaluated
by the library's operator application.  A step is one apply and one solve (Algorithm 2)
of a whole batch of initial conditions.
"""
import torch


def cn_coefficients(n_leaf, p, eps, k, device="cuda"):
    """Coefficient fields (6, n_leaf, p*p) of I/k - A/2 with A = eps Laplace - d/dx."""
    c = torch.zeros((6, n_leaf, p * p), dtype=torch.float64, device=device)
    c[0] = eps / 2
    c[2] = eps / 2
    c[3] = 0.5
    c[5] = 1.0 / k
    return c


def channel_solver(tree, p, eps, k, **kw):
    """The built step operator on a periodic channel (periodic west/east, Neumann
    south/north) and its coefficient fields."""
    from .solver import Solver
    n_leaf = tree.info(p - 1)["n_leaves"]
    coeffs = cn_coefficients(n_leaf, p, eps, k)
    return Solver(tree, coeffs, p, "fp64", bc_we="periodic", bc_sn="neumann", **kw), coeffs


def crank_nicolson(solver, coeffs, u0, k, nsteps, flux=None, callback=None):
    """Advance u0 (n_leaf, p*p[, nrhs]) by nsteps Crank-Nicolson steps of size k.  flux:
    du/dy data at the south/north boundary nodes (zero when None), shaped like the
    solver's f.  callback(n, u), if given, runs after every step."""
    u = u0
    squeeze = u.dim() == 2
    nrhs = 1 if squeeze else u.shape[-1]
    if flux is None:
        flux = torch.zeros((solver.n_bdry,) if squeeze else (solver.n_bdry, nrhs), dtype=torch.float64,
                           device=u.device)
    for n in range(nsteps):
        g = solver.apply(coeffs, u, 2.0 / k, -1.0)
        u = solver.solve(flux, g)
        if callback is not None:
            callback(n + 1, u)
    return u
