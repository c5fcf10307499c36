"""GPU parity at the benchmark's own sizes, element by element against the oracle.

* The variable-coefficient workload: 64 x 64 leaves, p = 16, seeded coefficient fields,
  64 distinct right-hand sides: the whole solution (every leaf Chebyshev node and every
  Gaussian node) of the FP64 path within 1e-10 and of the mixed path within 1e-8, relative
  l-infinity, at nrhs 64 and 1.
* Constant-coefficient Poisson on 4 x 4 leaves, p = 16, with the manufactured solution
  u* = sin(pi x) sin(2 pi y) + x^2 y: against the oracle and against u*.
* Higher orders p = 24 and p = 30 (8 x 8 leaves; leaf systems of 596 and 900 unknowns, so
  the products with inner dimension above 448 take the SIMT path), FP64 and mixed.
* The backward-Euler operator on 128 x 128 leaves, p = 16 (dt = 1e-3): the eigenmode
  closed form over 10 steps, and one step of the seeded Gaussian ensemble checked against
  the discrete equations on every leaf and every interior edge with the oracle's dense
  leaf operators."""
import numpy as np
import pytest

import synthetic as syn
from oracle import hps, leaf as lfm, spectral as sp, tree as tr
from tests.gpu_common import gpu_tree, make_case, oracle_solve, to_dev
from tests.helpers import boundary_points, leaf_points, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def varcoef64():
    """The 64 x 64, p = 16 workload with 64 right-hand sides and the oracle's solution."""
    case = make_case(64, 64, 16, nrhs=64)
    (uc, ug), _ = oracle_solve(case)
    return case, uc, ug


def _gpu_solve(case, precision, nrhs, **kw):
    from paper_1612_02736_gb300 import Solver
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), case["p"], precision=precision, **kw)
    f = to_dev(case["f"][:, :nrhs])
    g = to_dev(case["g"][..., :nrhs])
    u, ug = s.solve(f, g, return_gauss=True)
    u2 = s.solve(f, g)  # a repeat solve (captured graph / calibrated refinement)
    out = u.cpu().numpy(), ug.cpu().numpy(), u2.cpu().numpy(), s.last_iters
    s.close()
    return out


@pytest.mark.parametrize("precision,nrhs", [("fp64", 64), ("fp64", 1), ("mixed", 64), ("mixed", 1)])
def test_varcoef_64x64_p16_whole_solution(varcoef64, precision, nrhs):
    case, uc, ug = varcoef64
    u, ugg, u2, _ = _gpu_solve(case, precision, nrhs)
    tol = 1e-10 if precision == "fp64" else 1e-8
    ref_c, ref_g = uc[..., :nrhs], ug[:, :nrhs]
    for got in (u, u2):
        assert rel_linf(got, ref_c) < tol, rel_linf(got, ref_c)
    assert rel_linf(ugg, ref_g) < tol


def test_poisson_4x4_p16_manufactured():
    case = make_case(4, 4, 16, kind="poisson", nrhs=1)  # the manufactured data, replicated
    case["f"] = np.repeat(case["f"], 64, axis=1)
    case["g"] = np.repeat(case["g"], 64, axis=2)
    (uc, ug), _ = oracle_solve(case)
    u_star = syn.u_star(case["X"], case["Y"])
    for precision, tol in (("fp64", 1e-10), ("mixed", 1e-8)):
        for nrhs in (1, 64):
            u, ugg, _, _ = _gpu_solve(case, precision, nrhs)
            assert rel_linf(u, uc[..., :nrhs]) < tol
            assert rel_linf(ugg, ug[:, :nrhs]) < tol
            # spectral accuracy of the discretisation itself (Sec. 7.1)
            assert np.max(np.abs(u - u_star[..., None])) < 1e-9


@pytest.mark.parametrize("p", [24, 30])
def test_high_order_8x8(p):
    case = make_case(8, 8, p, nrhs=16)
    (uc, ug), _ = oracle_solve(case)
    for precision, tol in (("fp64", 1e-10), ("mixed", 1e-8)):
        for nrhs in (1, 16):
            u, ugg, u2, _ = _gpu_solve(case, precision, nrhs)
            assert rel_linf(u, uc[..., :nrhs]) < tol, (precision, nrhs, rel_linf(u, uc[..., :nrhs]))
            assert rel_linf(u2, uc[..., :nrhs]) < tol
            assert rel_linf(ugg, ug[:, :nrhs]) < tol


def _equation_residuals(t, p, coeffs_leaf, u, ug, g, f):
    """Discrete equations of the collocation system on every leaf of a uniform tree whose
    leaves share one operator: (collocation residual, flux jump, boundary mismatch,
    exterior-value mismatch), each relative to the size of the terms that cancel in it."""
    q = p - 1
    ce, ci, _ = sp.leaf_index_sets(p)
    x0, y0, x1, y1 = t.leaf_rect(0)
    A = lfm.leaf_A(coeffs_leaf, p, x1 - x0, y1 - y0)
    L = sp.L_ce_ge(p, q)
    Dg = sp.D_ge_c(p, q, x1 - x0, y1 - y0)
    ge = np.array([t.boxes[t.leaves[lf]].ge for lf in range(t.n_leaves)])
    ext = np.einsum("ij,ljr->lir", L, ug[ge])
    e_ext = np.max(np.abs(u[:, ce] - ext)) / np.max(np.abs(u))
    Au = np.einsum("ij,ljr->lir", A[ci], u)
    Aabs = np.einsum("ij,ljr->lir", np.abs(A[ci]), np.abs(u))
    e_col = np.max(np.abs(g[:, ci] - Au)) / np.max(Aabs)
    v = np.einsum("ij,ljr->lir", Dg, u)
    vabs = np.einsum("ij,ljr->lir", np.abs(Dg), np.abs(u))
    pr = t.interior_pairs
    e_jump = np.max(np.abs(v[pr[:, 0], pr[:, 1]] - v[pr[:, 2], pr[:, 3]])) / np.max(vabs)
    e_bnd = np.max(np.abs(ug[t.boundary] - f)) / np.max(np.abs(f))
    return e_col, e_jump, e_bnd, e_ext


def test_heat_operator_128x128_p16():
    import torch
    from paper_1612_02736_gb300 import Solver, Tree
    from paper_1612_02736_gb300.heat import backward_euler, heat_coefficients
    n, p, dt = 128, 16, 1e-3
    t = tr.uniform_tree(0.0, 0.0, 1.0, 1.0, n, n, p - 1)
    X, Y = leaf_points(t, p)
    bx, by = boundary_points(t)
    gt = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    coeffs = heat_coefficients(n * n, p, dt)
    coeffs_leaf = [coeffs[k, 0].cpu().numpy() for k in range(6)]
    # (a) eigenmode: u^n = (1 + 2 pi^2 dt)^-n sin(pi x) sin(pi y) up to spatial error
    s = Solver(gt, coeffs, p, "fp64")
    u0 = np.sin(np.pi * X) * np.sin(np.pi * Y)
    zero = torch.zeros(s.n_bdry, dtype=torch.float64, device="cuda")
    u = backward_euler(s, to_dev(u0), lambda tt: zero, dt, 10)
    expect = (1 + 2 * np.pi ** 2 * dt) ** (-10) * u0
    assert np.max(np.abs(u.cpu().numpy() - expect)) < 1e-9
    # (b) one step of four seeded ensemble members with f = sin(t) x y: the discrete
    # equations on every leaf and interior edge, per-leaf operators (no leaf sharing) for
    # FP64 and for the mixed path
    members = 4
    u0 = np.stack([syn.heat_initial(X, Y, member=k) for k in range(members)], axis=-1)
    f = np.repeat((np.sin(dt) * bx * by)[:, None], members, axis=1)
    for precision, tol in (("fp64", 1e-13), ("mixed", 1e-8)):
        s = Solver(gt, coeffs, p, precision, shared_leaf=False)
        u1, ug1 = s.solve(to_dev(f), to_dev(u0), return_gauss=True)
        res = _equation_residuals(t, p, coeffs_leaf, u1.cpu().numpy(), ug1.cpu().numpy(), u0, f)
        assert max(res) < tol, (precision, res)
        s.close()
