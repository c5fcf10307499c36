"""GPU parity on locally refined trees and the L-shaped domain (Sec. 6): the CUDA build,
solve and adjoint with the coarse-fine interpolation steps against the CPU oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import hps, tree as tr
from tests.gpu_common import to_dev
from tests.helpers import boundary_points, leaf_points, poly_data, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


def _pair(kind, p):
    from paper_1612_02736_gb300 import Tree
    q = p - 1
    if kind[0] == "uniform":
        _, nx, ny, pts, lev = kind
        o = tr.refine_tree(tr.uniform_tree(0, 0, 1, 1, nx, ny, q), pts, lev)
        g = Tree.uniform(0.0, 0.0, 1.0, 1.0, nx, ny).refine(pts, lev)
    else:
        _, n, pts, lev = kind
        o = tr.refine_tree(tr.l_shape_tree(n, q), pts, lev)
        g = Tree.l_shape(n).refine(pts, lev)
    return o, g


CASES = [("uniform", 3, 3, [(0.1, 0.9)], 2), ("uniform", 6, 3, [(0.6, 0.2), (0.05, 0.95)], 1),
         ("uniform", 4, 2, [(0.6, 0.1)], 2), ("lshape", 2, [(0.0, 0.0)], 3)]


@pytest.mark.parametrize("kind", CASES)
@pytest.mark.parametrize("p,nrhs", [(8, 1), (9, 6)])
def test_refined_fp64_matches_oracle(kind, p, nrhs):
    from paper_1612_02736_gb300 import Solver
    o, gt = _pair(kind, p)
    X, Y = leaf_points(o, p)
    prob = syn.VarCoeffProblem()
    coeffs = np.array(prob.coeffs(X, Y))
    bx, by = boundary_points(o)
    sc = np.linspace(0.5, 1.5, nrhs)
    g = prob.load(X, Y)[..., None] * sc
    f = prob.dirichlet(bx, by)[:, None] * sc
    rho = np.random.default_rng(3).standard_normal((o.n_gauss, nrhs))
    ops = hps.build(o, coeffs, p)
    uc, ug = hps.solve(o, ops, p, f, g, rho)
    s = Solver(gt, to_dev(coeffs), p)
    u, ugg = s.solve(to_dev(f), to_dev(g), rho=to_dev(rho), return_gauss=True)
    assert rel_linf(u.cpu().numpy(), uc) < 1e-10
    assert rel_linf(ugg.cpu().numpy(), ug) < 1e-10
    # polynomial exactness through every coarse-fine interface
    up, gp = poly_data(X, Y, coeffs, p - 2, 3)
    u2 = s.solve(to_dev(bx ** (p - 2) * by ** 3), to_dev(gp))
    assert np.max(np.abs(u2.cpu().numpy() - up)) < 1e-9
    # adjoint
    ubar = np.random.default_rng(4).standard_normal(uc.shape)
    fb, gb, _ = hps.adjoint(o, ops, p, ubar)
    cg = hps.coeff_gradients(o, p, uc, gb)
    u0 = s.solve(to_dev(f), to_dev(g))
    fbg, gbg, cgg = s.adjoint(to_dev(ubar), u=to_dev(hps.solve(o, ops, p, f, g)[0]))
    assert rel_linf(fbg.cpu().numpy(), fb) < 1e-9
    assert rel_linf(gbg.cpu().numpy(), gb) < 1e-9
    del u0


def test_lshape_config_full_size():
    # The locally refined L-shape workload: 32 x 32 base squares over [-1,1]^2 minus the
    # south-east quadrant, 5 levels of refinement toward the re-entrant corner and a seeded
    # point-load centre, p = 20, Laplace operator; compared with the oracle everywhere.
    from paper_1612_02736_gb300 import Solver
    p = 20
    c = syn.lshape_load_centre()
    o, gt = _pair(("lshape", 16, [(0.0, 0.0), c], 5), p)
    X, Y = leaf_points(o, p)
    n = X.shape
    coeffs = np.array([np.ones(n), np.zeros(n), np.ones(n), np.zeros(n), np.zeros(n), np.zeros(n)])
    bx, by = boundary_points(o)
    th = np.mod(np.arctan2(by, bx), 2 * np.pi)
    f = np.stack([np.hypot(bx, by) ** (2.0 / 3.0) * np.sin(2.0 * th / 3.0), np.zeros_like(bx)], axis=1)
    g = np.stack([np.zeros(n), syn.point_load(X, Y, c)], axis=-1)
    uc, _ = hps.solve(o, hps.build(o, coeffs, p), p, f, g)
    s = Solver(gt, to_dev(coeffs), p)
    u = s.solve(to_dev(f), to_dev(g)).cpu().numpy()
    assert rel_linf(u[..., 0], uc[..., 0]) < 1e-10
    assert np.max(np.abs(u[..., 1] - uc[..., 1])) < 1e-10 * max(np.max(np.abs(uc[..., 1])), 1e-3)
