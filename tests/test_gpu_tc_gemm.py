"""FP64 solve and adjoint products on the tensor cores by exact digit slicing, through the
C ABI: against the CPU oracle (FP64 tolerance) and against the SIMT FP64 products of the
same build, on problems whose leaf products have inner dimension up to 400 (tensor-core
eligible, up to 448) and above (the SIMT fallback), with ragged right-hand-side blocks."""
import numpy as np
import pytest

from oracle import hps
from tests.gpu_common import gpu_tree, make_case, oracle_solve, to_dev
from tests.helpers import rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


# leaf products: K = (p - 2)^2 + 4 (p - 1): 256 at p = 16, 400 at p = 20, 484 at p = 22 (> 448)
@pytest.mark.parametrize("nx,ny,p,nrhs", [(4, 4, 16, 8), (3, 2, 12, 33), (2, 2, 20, 64), (2, 1, 22, 16),
                                          (8, 8, 10, 40)])
def test_tensor_products_match_oracle_and_simt(nx, ny, p, nrhs):
    from paper_1612_02736_gb300 import Solver
    case = make_case(nx, ny, p, nrhs=nrhs)
    (uc, ug), ops = oracle_solve(case)
    res = {}
    for path in ("tensor", "simt"):
        s = Solver(gpu_tree(case), to_dev(case["coeffs"]), p, fp64_gemm=path)
        u, ugg = s.solve(to_dev(case["f"]), to_dev(case["g"]), return_gauss=True)
        res[path] = (u.cpu().numpy(), ugg.cpu().numpy())
        assert rel_linf(res[path][0], uc) < 1e-10
        assert rel_linf(res[path][1], ug) < 1e-10
    # the two paths agree to FP64 rounding of the products
    assert rel_linf(res["tensor"][0], res["simt"][0]) < 1e-12


@pytest.mark.parametrize("nx,ny,p,nrhs", [(4, 4, 16, 8), (2, 2, 20, 24)])
def test_tensor_products_adjoint_matches_oracle(nx, ny, p, nrhs):
    from paper_1612_02736_gb300 import Solver
    case = make_case(nx, ny, p, nrhs=nrhs)
    (uc, _), ops = oracle_solve(case)
    ubar = np.random.default_rng(5).standard_normal(uc.shape)
    fb, gb, _ = hps.adjoint(case["tree"], ops, p, ubar)
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), p, fp64_gemm="tensor")
    fbg, gbg, _ = s.adjoint(to_dev(ubar), want_coeffs=False)
    assert rel_linf(fbg.cpu().numpy(), fb) < 1e-9
    assert rel_linf(gbg.cpu().numpy(), gb) < 1e-9


def test_tensor_products_econ_and_graphs_off():
    # operators rebuilt chunk by chunk (econ) and direct launches instead of the captured sweep
    from paper_1612_02736_gb300 import Solver
    case = make_case(8, 8, 16, nrhs=16)
    (uc, _), _ = oracle_solve(case)
    for kw in ({"store_leaf_ops": False}, {"use_graphs": False}):
        s = Solver(gpu_tree(case), to_dev(case["coeffs"]), 16, fp64_gemm="tensor", **kw)
        u = s.solve(to_dev(case["f"]), to_dev(case["g"]))
        assert rel_linf(u.cpu().numpy(), uc) < 1e-10


def test_cached_operator_digits_reproduce_the_first_solve():
    # The first solve forms the operators' digits inside the products; the second (captured
    # into a graph) and later solves read the cached digit planes.  Same digits, same
    # arithmetic: results bit for bit equal.  The adjoint likewise on its second call.
    import torch
    from paper_1612_02736_gb300 import Solver
    case = make_case(8, 8, 16, nrhs=16)
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), 16)
    f, g = to_dev(case["f"]), to_dev(case["g"])
    u1 = s.solve(f, g)
    u2 = s.solve(f, g)
    u3 = s.solve(f, g)
    assert torch.equal(u1, u2) and torch.equal(u1, u3)
    ubar = to_dev(np.random.default_rng(3).standard_normal(case["g"].shape))
    a1 = s.adjoint(ubar, want_coeffs=False)
    a2 = s.adjoint(ubar, want_coeffs=False)
    assert torch.equal(a1[0], a2[0]) and torch.equal(a1[1], a2[1])
