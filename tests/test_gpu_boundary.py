"""Periodic and Neumann root conditions on the GPU (Sec. 7.6) against the oracle, the
closed-form periodic channel, and Crank-Nicolson stepping of the convection-diffusion
problem (the library's operator application plus one solve per step)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import boundary as bd, hps, leaf as lfm, tree as tr
from tests.gpu_common import to_dev
from tests.helpers import boundary_points, leaf_points, rel_linf

pytestmark = pytest.mark.gpu

KINDS = {(bd.PERIODIC, bd.NEUMANN): ("periodic", "neumann"), (bd.PERIODIC, bd.DIRICHLET): ("periodic", "dirichlet"),
         (bd.DIRICHLET, bd.NEUMANN): ("dirichlet", "neumann")}


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


@pytest.mark.parametrize("bc", list(KINDS))
@pytest.mark.parametrize("nx,ny,p", [(1, 1, 8), (2, 2, 8), (4, 2, 7), (8, 8, 12), (5, 3, 9)])
def test_root_conditions_match_oracle(bc, nx, ny, p):
    import torch
    from paper_1612_02736_gb300 import Solver, Tree
    o = tr.uniform_tree(0, 0, 1, 1, nx, ny, p - 1)
    X, Y = leaf_points(o, p)
    bx, by = boundary_points(o)
    prob = syn.VarCoeffProblem()
    coeffs = np.array(prob.coeffs(X, Y))
    coeffs[5] += 1.0
    g = np.stack([prob.load(X, Y), np.cos(2 * X) * Y], axis=-1)
    f = np.stack([np.sin(3 * bx) + by, bx * by], axis=-1)
    uc, _ = hps.solve(o, hps.build(o, coeffs, p), p, f, g, bc=bc)
    we, sn = KINDS[bc]
    s = Solver(Tree.uniform(0.0, 0.0, 1.0, 1.0, nx, ny), to_dev(coeffs), p, bc_we=we, bc_sn=sn)
    fd, gd = to_dev(f), to_dev(g)
    u1 = s.solve(fd, gd)
    assert rel_linf(u1.cpu().numpy(), uc) < 1e-10
    u2 = s.solve(fd, gd)          # second call: the captured sweep replays
    assert torch.equal(u1, u2)


def test_periodic_channel_closed_form():
    from paper_1612_02736_gb300 import Solver, Tree
    eps, k, n, p = 1 / 200, 1e-2, 16, 16
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    xy = t.nodes(p, p - 1, "cheb")
    X, Y = xy[:, 0].reshape(n * n, p * p), xy[:, 1].reshape(n * n, p * p)
    z = np.zeros_like(X)
    coeffs = np.array([z + eps / 2, z, z + eps / 2, z + 0.5, z, z + 1 / k])
    u = np.cos(2 * np.pi * X) * np.cos(np.pi * Y)
    g = (eps / 2) * 5 * np.pi ** 2 * u + 0.5 * (-2 * np.pi * np.sin(2 * np.pi * X) * np.cos(np.pi * Y)) + u / k
    s = Solver(t, to_dev(coeffs), p, bc_we="periodic", bc_sn="neumann")
    uh = s.solve(to_dev(np.zeros(s.n_bdry)), to_dev(g)).cpu().numpy()
    assert np.max(np.abs(uh - u)) < 1e-9


def test_apply_matches_oracle():
    import torch
    from paper_1612_02736_gb300 import Solver, Tree
    n, p = 4, 12
    o = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(o, p)
    coeffs = np.array(syn.VarCoeffProblem().coeffs(X, Y))
    u = np.stack([np.sin(X + k) * np.exp(Y) for k in range(3)], axis=-1)
    s = Solver(Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n), to_dev(coeffs), p)
    y = s.apply(to_dev(coeffs), to_dev(u), 0.5, -2.0).cpu().numpy()
    _, ci, _ = __import__("oracle.spectral", fromlist=["x"]).leaf_index_sets(p)
    for lf in range(n * n):
        A = lfm.leaf_A(coeffs[:, lf], p, 1 / n, 1 / n)
        expect = 0.5 * u[lf] - 2.0 * A @ u[lf]
        # rounding of a sum of products is relative to |A| |u| (spectral second
        # derivatives cancel heavily): double-float unit roundoff is about 3.6e-15
        scale = 0.5 * np.max(np.abs(u[lf])) + 2.0 * np.max(np.abs(A).sum(axis=1)) * np.max(np.abs(u[lf]))
        assert np.max(np.abs(y[lf][ci] - expect[ci])) < 1e-13 * scale
        mask = np.ones(p * p, bool)
        mask[ci] = False
        assert np.all(y[lf][mask] == 0.0)
    torch.cuda.synchronize()


def test_crank_nicolson_channel_matches_oracle():
    # The convection-diffusion problem of Sec. 7.6: eps = 1/200, u0 a Gaussian (alpha = 50)
    # at (1/4, 1/4), 16 x 16 leaves with q = 16 (p = 17), step k = 1e-2, 10 steps.
    import torch
    from paper_1612_02736_gb300 import Tree
    from paper_1612_02736_gb300.convdiff import channel_solver, crank_nicolson
    eps, k, n, p, steps = 1 / 200, 1e-2, 16, 17, 10
    o = tr.uniform_tree(0, 0, 1, 1, n, n, p - 1)
    X, Y = leaf_points(o, p)
    bx, _ = boundary_points(o)
    u0 = np.exp(-50.0 * ((X - 0.25) ** 2 + (Y - 0.25) ** 2))
    z = np.zeros_like(X)
    M = np.array([z + eps / 2, z, z + eps / 2, z + 0.5, z, z + 1 / k])
    ops = hps.build(o, M, p)
    uo = u0
    for _ in range(steps):
        Mu = np.array([lfm.apply_A(M[:, lf], uo[lf], p, 1 / n, 1 / n) for lf in range(n * n)])
        uo = hps.solve(o, ops, p, np.zeros_like(bx), (2 / k) * uo - Mu, bc=(bd.PERIODIC, bd.NEUMANN))[0][..., 0]
    s, coeffs = channel_solver(Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n), p, eps, k)
    u = crank_nicolson(s, coeffs, to_dev(u0), k, steps).cpu().numpy()
    assert rel_linf(u, uo) < 1e-10
    torch.cuda.synchronize()


def test_crank_nicolson_fourier_mode():
    from paper_1612_02736_gb300 import Tree
    from paper_1612_02736_gb300.convdiff import channel_solver, crank_nicolson
    eps, k, n, p, steps = 1 / 200, 2e-2, 4, 16, 5
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    xy = t.nodes(p, p - 1, "cheb")
    X, Y = xy[:, 0].reshape(n * n, p * p), xy[:, 1].reshape(n * n, p * p)
    s, coeffs = channel_solver(t, p, eps, k)
    u = crank_nicolson(s, coeffs, to_dev(np.cos(2 * np.pi * X) * np.cos(np.pi * Y)), k, steps).cpu().numpy()
    lam = -5 * np.pi ** 2 * eps - 2j * np.pi
    G = (1 / k + lam / 2) / (1 / k - lam / 2)
    exact = np.real(G ** steps * np.exp(2j * np.pi * X)) * np.cos(np.pi * Y)
    assert np.max(np.abs(u - exact)) < 1e-9


def test_root_conditions_reject_other_paths():
    import torch
    from paper_1612_02736_gb300 import Solver, Tree, _native
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, 2, 2)
    c = torch.zeros((6, 4, 64), dtype=torch.float64, device="cuda")
    c[0] = 1.0
    c[2] = 1.0
    c[5] = 1.0
    with pytest.raises(_native.HPSError) as e:
        Solver(t, c, 8, "mixed", bc_we="periodic")
    assert e.value.code == 1
    s = Solver(t, c, 8, bc_sn="neumann")
    u = s.solve(torch.zeros(s.n_bdry, dtype=torch.float64, device="cuda"), torch.ones((4, 64), dtype=torch.float64,
                                                                                      device="cuda"))
    with pytest.raises(_native.HPSError) as e:
        s.adjoint(u, u=u)
    assert e.value.code == 8
