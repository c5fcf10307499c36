"""Implicit time stepping with a fixed solution operator (Sec. 1, Eq. heat; Sec. 7.6).

Backward Euler for u_t = Laplace(u): each step solves (I - dt Laplace) u^{n+1} = u^n, i.e.
Eq. basic with c11 = c22 = dt, c = 1 (other coefficients zero), load g = u^n and the
boundary data of the new time.  The operator is built once (Algorithm 1) and every step is
one solve (Algorithm 2) of a whole ensemble of initial conditions, so the per-step work
is the sweep kernels only.
"""
import torch


def heat_coefficients(n_leaf, p, dt, device="cuda"):
    """Coefficient fields (6, n_leaf, p*p) of I - dt Laplace."""
    c = torch.zeros((6, n_leaf, p * p), dtype=torch.float64, device=device)
    c[0] = dt
    c[2] = dt
    c[5] = 1.0
    return c


def backward_euler(solver, u0, boundary, dt, nsteps, t0=0.0, callback=None):
    """Advance u0 (n_leaf, p*p[, nrhs]) by nsteps of size dt.  boundary(t) returns the
    Dirichlet data at the boundary Gaussian nodes for time t, shaped like the solver's f.
    callback(n, t, u), if given, is called after every step."""
    u = u0
    t = t0
    for n in range(nsteps):
        t = t0 + (n + 1) * dt
        u = solver.solve(boundary(t), u)
        if callback is not None:
            callback(n + 1, t, u)
    return u
