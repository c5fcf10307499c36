"""Shared set-up of the GPU tests: problems are generated from oracle coordinates and the
``synthetic`` module, solved by the oracle on the CPU and by the library on the GPU."""
import numpy as np

import synthetic as syn
from oracle import hps, tree as tr
from tests.helpers import boundary_points, leaf_points


def make_case(nx, ny, p, kind="var", rect=(0.0, 0.0, 1.0, 1.0), nrhs=1, seed=0):
    q = p - 1
    t = tr.uniform_tree(*rect, nx, ny, q)
    X, Y = leaf_points(t, p)
    bx, by = boundary_points(t)
    if kind == "var":
        prob = syn.VarCoeffProblem(box=rect)
        coeffs = np.array(prob.coeffs(X, Y))
        g0, f0 = prob.load(X, Y), prob.dirichlet(bx, by)
    else:
        c, g0 = syn.poisson_manufactured(X, Y)
        coeffs = np.array(c)
        f0 = syn.u_star(bx, by)
    rng = np.random.default_rng(100 + seed)
    g = np.repeat(g0[..., None], nrhs, axis=-1)
    f = np.repeat(f0[:, None], nrhs, axis=-1)
    if nrhs > 1:  # distinct right-hand sides: scaled copies plus smooth perturbations
        sc = rng.uniform(0.5, 1.5, nrhs)
        g = g * sc + 0.1 * np.sin(np.arange(nrhs) + X[..., None] * 3.0) * np.cos(Y[..., None] * 2.0)
        f = f * sc + 0.1 * np.cos(np.arange(nrhs) + bx[:, None] * 2.0) * by[:, None]
    return {"tree": t, "coeffs": coeffs, "g": g, "f": f, "X": X, "Y": Y, "p": p, "rect": rect, "nx": nx, "ny": ny}


def oracle_solve(case, rho=None):
    ops = hps.build(case["tree"], case["coeffs"], case["p"])
    return hps.solve(case["tree"], ops, case["p"], case["f"], case["g"], rho), ops


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def gpu_tree(case):
    from paper_1612_02736_gb300 import Tree
    return Tree.uniform(*case["rect"], case["nx"], case["ny"])
