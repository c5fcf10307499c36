"""Backward-Euler heat stepping with one operator built once: the eigenmode closed form
(pin P12) and the oracle's step-by-step result, in FP64 and in mixed precision."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_heat_eigenmode(precision):
    # u^0 = sin(pi x) sin(pi y), f = 0: u^n = (1 + 2 pi^2 dt)^-n u^0 up to spatial error.
    import torch
    from paper_1612_02736_gb300 import Solver, Tree
    from paper_1612_02736_gb300.heat import backward_euler, heat_coefficients
    n, p, dt, steps = 16, 16, 1e-3, 25
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    xy = t.nodes(p, p - 1, "cheb")
    X, Y = xy[:, 0].reshape(n * n, p * p), xy[:, 1].reshape(n * n, p * p)
    s = Solver(t, heat_coefficients(n * n, p, dt), p, precision=precision)
    u0 = to_dev(np.sin(np.pi * X) * np.sin(np.pi * Y))
    zero = torch.zeros(s.n_bdry, dtype=torch.float64, device="cuda")
    u = backward_euler(s, u0, lambda tt: zero, dt, steps)
    expect = (1 + 2 * np.pi ** 2 * dt) ** (-steps) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    assert np.max(np.abs(u.cpu().numpy() - expect)) < 1e-9


def test_heat_ensemble_matches_oracle():
    # 4 ensemble members (seeded Gaussian sums), f = sin(t) x y, 5 steps: GPU mixed and FP64
    # against the oracle stepping the same system.
    import torch
    from paper_1612_02736_gb300 import Solver, Tree
    from paper_1612_02736_gb300.heat import backward_euler, heat_coefficients
    n, p, dt, steps, members = 4, 12, 1e-3, 5, 4
    o = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(o, p)
    bx, by = boundary_points(o)
    u0 = np.stack([syn.heat_initial(X, Y, member=k) for k in range(members)], axis=-1)
    coeffs = heat_coefficients(n * n, p, dt, device="cpu").numpy()
    ops = hps.build(o, coeffs, p)
    uo = u0
    for k in range(steps):
        tk = (k + 1) * dt
        uo = hps.solve(o, ops, p, np.repeat((np.sin(tk) * bx * by)[:, None], members, 1), uo)[0]
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    bxy = to_dev(bx * by)
    for precision in ("fp64", "mixed"):
        s = Solver(t, heat_coefficients(n * n, p, dt), p, precision=precision)
        u = backward_euler(s, to_dev(u0), lambda tt: (np.sin(tt) * bxy)[:, None].repeat(1, members), dt, steps)
        assert rel_linf(u.cpu().numpy(), uo) < (1e-10 if precision == "fp64" else 1e-8)
    torch.cuda.synchronize()
