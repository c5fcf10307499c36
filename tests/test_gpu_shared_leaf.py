"""Leaf operators shared by every leaf when all leaves are equal (the constant-coefficient
remark of Sec. 7.1): one leaf is eliminated and stored, and the build, solve and adjoint
agree with the per-leaf operators and with the oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import hps, tree as tr
from tests.gpu_common import to_dev
from tests.helpers import boundary_points, leaf_points, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


def _constant_case(n, p, nrhs):
    o = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(o, p)
    bx, by = boundary_points(o)
    z = np.zeros_like(X)
    # constant anisotropic operator with drift and reaction
    coeffs = np.array([z + 1.3, z + 0.2, z + 0.7, z + 0.5, z - 0.4, z + 2.0])
    g = np.stack([np.sin(3 * X + k) * np.cos(2 * Y) for k in range(nrhs)], axis=-1)
    f = np.stack([np.cos(bx + k) * by for k in range(nrhs)], axis=-1)
    return o, coeffs, f, g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shared_matches_per_leaf_and_oracle(precision):
    import torch
    from paper_1612_02736_gb300 import Solver, Tree
    n, p, nrhs = 8, 12, 3
    o, coeffs, f, g = _constant_case(n, p, nrhs)
    (uc, _), = [hps.solve(o, hps.build(o, coeffs, p), p, f, g)]
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    sa = Solver(t, to_dev(coeffs), p, precision)                      # auto: shared
    sb = Solver(t, to_dev(coeffs), p, precision, shared_leaf=False)   # per leaf
    m, nq = (p - 2) ** 2, 4 * (p - 1)
    per_leaf = (m * (m + nq) + nq * m) * (8 if precision == "fp64" else 4)   # [F | S_ci] and H
    assert sb.operator_bytes - sa.operator_bytes == (n * n - 1) * per_leaf
    ua = sa.solve(to_dev(f), to_dev(g)).cpu().numpy()
    ub = sb.solve(to_dev(f), to_dev(g)).cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert rel_linf(ua, uc) < tol
    assert rel_linf(ua, ub) < (1e-12 if precision == "fp64" else 1e-8)
    torch.cuda.synchronize()


def test_shared_adjoint_matches_per_leaf():
    from paper_1612_02736_gb300 import Solver, Tree
    n, p, nrhs = 4, 10, 2
    o, coeffs, f, g = _constant_case(n, p, nrhs)
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    sa = Solver(t, to_dev(coeffs), p, shared_leaf=True)
    sb = Solver(t, to_dev(coeffs), p, shared_leaf=False)
    u = sb.solve(to_dev(f), to_dev(g))
    ubar = to_dev(np.random.default_rng(5).standard_normal(g.shape))
    ra = sa.adjoint(ubar, u=u)
    rb = sb.adjoint(ubar, u=u)
    for x, y in zip(ra, rb):
        assert rel_linf(x.cpu().numpy(), y.cpu().numpy()) < 1e-12


def test_varying_coefficients_are_not_shared():
    import torch
    from paper_1612_02736_gb300 import Solver, Tree, _native
    n, p = 4, 8
    o, coeffs, f, g = _constant_case(n, p, 1)
    coeffs = coeffs.copy()
    coeffs[5, 7, 20] += 1e-3    # one interior value of one leaf differs
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    sa = Solver(t, to_dev(coeffs), p)
    sb = Solver(t, to_dev(coeffs), p, shared_leaf=False)
    assert sa.operator_bytes == sb.operator_bytes
    with pytest.raises(_native.HPSError):
        Solver(t, to_dev(coeffs), p, shared_leaf=True)
    (uc, _) = hps.solve(o, hps.build(o, coeffs, p), p, f, g)
    assert rel_linf(sa.solve(to_dev(f), to_dev(g)).cpu().numpy(), uc) < 1e-10
    # an exterior value may differ: the method never reads it, the leaves stay shared
    c2 = coeffs.copy()
    c2[5, 7, 20] -= 1e-3
    c2[0, 3, 0] = 5.0
    assert Solver(t, to_dev(c2), p).operator_bytes < sb.operator_bytes
    torch.cuda.synchronize()
