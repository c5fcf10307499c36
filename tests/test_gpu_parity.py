"""GPU parity: the CUDA build and solve (through the C ABI) against the CPU oracle,
element by element, on seeded inputs; FP64 within 1e-10 relative l-infinity, the mixed
FP32 + FP64-refinement path within 1e-8."""
import numpy as np
import pytest

from oracle import hps, leaf as lfm, spectral as sp
from tests.gpu_common import gpu_tree, make_case, oracle_solve, to_dev
from tests.helpers import boundary_points, poly_data, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


def run_gpu(case, precision="fp64", nrhs_squeeze=False, rho=None, **kw):
    from paper_1612_02736_gb300 import Solver
    t = gpu_tree(case)
    s = Solver(t, to_dev(case["coeffs"]), case["p"], precision=precision, **kw)
    u, ug = s.solve(to_dev(case["f"]), to_dev(case["g"]), rho=None if rho is None else to_dev(rho), return_gauss=True)
    return u.cpu().numpy(), ug.cpu().numpy(), s


@pytest.mark.parametrize("nx,ny,p,nrhs", [(1, 1, 8, 1), (2, 1, 8, 2), (2, 2, 10, 3), (3, 2, 8, 1),
                                          (4, 4, 12, 8), (5, 3, 9, 20), (8, 8, 16, 1), (4, 4, 16, 64)])
def test_fp64_matches_oracle(nx, ny, p, nrhs):
    case = make_case(nx, ny, p, nrhs=nrhs)
    (uc, ug), _ = oracle_solve(case)
    u, ugg, _ = run_gpu(case)
    assert rel_linf(u, uc) < 1e-10
    assert rel_linf(ugg, ug) < 1e-10


def test_rectangular_leaves_and_domain():
    case = make_case(4, 2, 10, rect=(-1.0, 0.5, 1.0, 1.0), nrhs=2)
    (uc, _), _ = oracle_solve(case)
    u, _, _ = run_gpu(case)
    assert rel_linf(u, uc) < 1e-10


def test_flux_jump_right_hand_side():
    case = make_case(4, 4, 10, nrhs=2)
    rho = np.random.default_rng(9).standard_normal((case["tree"].n_gauss, 2))
    (uc, ug), _ = oracle_solve(case, rho)
    u, ugg, _ = run_gpu(case, rho=rho)
    assert rel_linf(u, uc) < 1e-10 and rel_linf(ugg, ug) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_polynomial_exactness_on_gpu(precision):
    # u = x^a y^b (a, b <= q-1) is reproduced to rounding by the discrete scheme.
    case = make_case(8, 8, 16)
    t = case["tree"]
    bx, by = boundary_points(t)
    u_ex, g = poly_data(case["X"], case["Y"], case["coeffs"], 7, 12)
    case["g"] = g[..., None]
    case["f"] = (bx ** 7 * by ** 12)[:, None]
    u, _, _ = run_gpu(case, precision)
    assert np.max(np.abs(u[..., 0] - u_ex)) < 1e-9


@pytest.mark.parametrize("nx,ny,p,nrhs", [(4, 4, 16, 1), (8, 8, 16, 8), (3, 5, 12, 2)])
def test_mixed_matches_oracle(nx, ny, p, nrhs):
    case = make_case(nx, ny, p, nrhs=nrhs)
    (uc, _), _ = oracle_solve(case)
    u, _, s = run_gpu(case, "mixed")
    assert rel_linf(u, uc) < 1e-8
    assert 1 <= s.last_iters <= 10


def test_mixed_fp64_top_levels_variants():
    case = make_case(8, 8, 12, nrhs=1)
    (uc, _), _ = oracle_solve(case)
    for top in (0, 2, 100):
        u, _, _ = run_gpu(case, "mixed", fp64_top_levels=top)
        assert rel_linf(u, uc) < 1e-8


def _sampled_residuals(case, u, ug, leaves):
    """Discrete equations checked leaf by leaf with the oracle's dense leaf operators:
    collocation residual on sampled leaves and flux continuity across their edges."""
    t, p = case["tree"], case["p"]
    q = p - 1
    ce, ci, _ = sp.leaf_index_sets(p)
    L = sp.L_ce_ge(p, q)
    # residuals are measured against the size of the terms that cancel in them:
    # max_i sum_j |A_ij u_j| for the collocation rows, max |D_ge,c| |u| for the fluxes
    worst_r, worst_j, ascale, vscale = 0.0, 0.0, 0.0, 0.0
    flux = {}
    for lf in leaves:
        b = t.boxes[t.leaves[lf]]
        x0, y0, x1, y1 = b.rect
        coeffs = [case["coeffs"][k][lf] for k in range(6)]
        A = lfm.leaf_A(coeffs, p, x1 - x0, y1 - y0)
        uc = u[lf].copy()
        assert np.max(np.abs(uc[ce] - L @ ug[b.ge])) < 1e-11 * max(1.0, np.max(np.abs(uc)))
        r = case["g"][lf][ci] - A[ci] @ uc
        worst_r = max(worst_r, np.max(np.abs(r)))
        ascale = max(ascale, np.max(np.abs(A[ci]) @ np.abs(uc)))
        Dg = sp.D_ge_c(p, q, x1 - x0, y1 - y0)
        flux[lf] = Dg @ uc
        vscale = max(vscale, np.max(np.abs(Dg) @ np.abs(uc)))
    for la, pa, lb, pb in t.interior_pairs:
        if la in flux and lb in flux:
            worst_j = max(worst_j, np.max(np.abs(flux[la][pa] - flux[lb][pb])))
    return worst_r / ascale, worst_j / vscale


@pytest.mark.parametrize("precision,nrhs", [("fp64", 1), ("mixed", 16)])
def test_full_size_64x64_p16(precision, nrhs):
    # The benchmark workload (64 x 64 leaves, p = 16): (a) polynomial exactness, (b) the
    # collocation and flux-continuity equations on sampled leaves (any-size properties).
    case = make_case(64, 64, 16, nrhs=nrhs)
    t = case["tree"]
    u, ug, _ = run_gpu(case, precision)
    rng = np.random.default_rng(4)
    leaves = set(rng.choice(t.n_leaves, 12, replace=False).tolist())
    for lf in list(leaves):  # add east and north neighbours so shared edges are covered
        if lf % 64 < 63:
            leaves.add(lf + 1)
        if lf // 64 < 63:
            leaves.add(lf + 64)
    for r in range(nrhs) if nrhs <= 2 else (0, nrhs - 1):
        sub = dict(case, g=case["g"][..., r])
        res, jump = _sampled_residuals(sub, u[..., r], ug[:, r], sorted(leaves))
        tol = 1e-13 if precision == "fp64" else 1e-11
        assert res < tol and jump < tol, (res, jump)
    bx, by = boundary_points(t)
    u_ex, g = poly_data(case["X"], case["Y"], case["coeffs"], 5, 9)
    case["g"] = np.repeat(g[..., None], nrhs, axis=-1)
    case["f"] = np.repeat((bx ** 5 * by ** 9)[:, None], nrhs, axis=-1)
    u, _, _ = run_gpu(case, precision)
    assert np.max(np.abs(u - u_ex[..., None])) < 1e-9


def test_graph_replay_matches_direct_launches():
    # The FP64 sweep is captured into a CUDA graph on the second solve with a given nrhs;
    # replays with new data, a different nrhs and a workspace regrowth must all agree with
    # direct launches.
    from paper_1612_02736_gb300 import Solver
    import torch
    case = make_case(8, 4, 12, nrhs=3)
    t = gpu_tree(case)
    a = Solver(t, to_dev(case["coeffs"]), 12, use_graphs=True)
    b = Solver(t, to_dev(case["coeffs"]), 12, use_graphs=False)
    f, g = to_dev(case["f"]), to_dev(case["g"])
    for scale in (1.0, 2.0, -0.5):                 # second and third calls replay the graph
        ua, ub = a.solve(scale * f, scale * g), b.solve(scale * f, scale * g)
        assert ((ua - ub).abs().max() / ub.abs().max()).item() < 1e-13
    for k in (1, 1, 5, 5, 3, 3):                   # other nrhs, regrowth, back again
        fk, gk = f[:, :1].repeat(1, k), g[..., :1].repeat(1, 1, k)
        ua, ub = a.solve(fk, gk), b.solve(fk, gk)
        assert ((ua - ub).abs().max() / ub.abs().max()).item() < 1e-13
    torch.cuda.synchronize()


def test_reused_tree_plan_matches_fresh_tree():
    # Builds on one tree reuse its host plan: new coefficients, both precisions and other
    # p on the same tree must give bit-identical results to builds on freshly made trees.
    from paper_1612_02736_gb300 import Solver
    import torch
    case = make_case(4, 8, 10, nrhs=2)
    case2 = make_case(4, 8, 10, nrhs=2, rect=(0.0, 0.0, 1.0, 1.0), seed=1)
    c2 = case2["coeffs"] * np.array([1.1, 0.5, 0.9, -1.0, 2.0, 1.5])[:, None, None]
    t = gpu_tree(case)
    f, g = to_dev(case["f"]), to_dev(case["g"])
    for prec in ("fp64", "mixed", "fp64"):
        for coeffs in (case["coeffs"], c2, case["coeffs"]):
            u_re = Solver(t, to_dev(coeffs), 10, prec).solve(f, g)
            u_new = Solver(gpu_tree(case), to_dev(coeffs), 10, prec).solve(f, g)
            assert torch.equal(u_re, u_new)
    # another p on the same tree, then back
    case8 = make_case(4, 8, 8, nrhs=1)
    u8 = Solver(t, to_dev(case8["coeffs"]), 8).solve(to_dev(case8["f"]), to_dev(case8["g"]))
    (uc, _), _ = oracle_solve(case8)
    assert rel_linf(u8.cpu().numpy(), uc) < 1e-10
    u_again = Solver(t, to_dev(case["coeffs"]), 10).solve(f, g)
    (uo, _), _ = oracle_solve(case)
    assert rel_linf(u_again.cpu().numpy(), uo) < 1e-10
