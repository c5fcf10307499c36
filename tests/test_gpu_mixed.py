"""Mixed precision (FP32 sweeps refined against the double-float residual of the
collocation system): repeated solves on one handle.  The build measures the contraction
bound of the refinement on a model problem; the first solve refines until the bound
predicts convergence and fixes the number of corrections, which later solves run without
a test in between (captured in a CUDA graph from the second such call), testing once;
solves with flux-jump data refine adaptively.  Every solve is held to the 1e-8 relative
l-infinity target against the oracle."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("use_graphs", [True, False])
@pytest.mark.parametrize("nrhs", [1, 5, 40])
def test_calibrated_repeat_solves(use_graphs, nrhs):
    from paper_1612_02736_gb300 import Solver
    case = make_case(8, 8, 16, nrhs=nrhs)
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), 16, precision="mixed", use_graphs=use_graphs)
    iters = []
    for k, scale in enumerate((1.0, -0.7, 2.5, 0.3)):
        sub = dict(case, f=scale * case["f"] + 0.1 * k, g=scale * case["g"] - 0.2 * k)
        (uc, _), _ = oracle_solve(sub)
        u = s.solve(to_dev(sub["f"]), to_dev(sub["g"]))
        assert rel_linf(u.cpu().numpy(), uc) < 1e-8, (k, rel_linf(u.cpu().numpy(), uc))
        iters.append(s.last_iters)
    # the build measured the contraction bound: the first solve stops as soon as the bound
    # predicts convergence and fixes the count that later solves run (one correction for
    # FP32 sweeps on this problem)
    assert all(1 <= n <= 2 for n in iters) and all(n == iters[1] for n in iters[1:]), iters
    assert iters[-1] <= iters[0], iters


def test_flux_jump_data_keeps_adaptive_refinement():
    # solves with flux-continuity data are refined adaptively (never the fixed schedule)
    from paper_1612_02736_gb300 import Solver
    case = make_case(4, 4, 12, nrhs=2)
    rho = np.random.default_rng(3).standard_normal((case["tree"].n_gauss, 2))
    (uc, ug), _ = oracle_solve(case, rho)
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), 12, precision="mixed")
    for _ in range(3):
        s.solve(to_dev(case["f"]), to_dev(case["g"]))  # calibrates the handle
    u, ugg = s.solve(to_dev(case["f"]), to_dev(case["g"]), rho=to_dev(rho), return_gauss=True)
    assert rel_linf(u.cpu().numpy(), uc) < 1e-8 and rel_linf(ugg.cpu().numpy(), ug) < 1e-8
    assert s.last_iters >= 2


@pytest.mark.parametrize("nx,ny,p,nrhs", [(8, 8, 16, 9), (8, 4, 12, 64), (4, 4, 10, 100)])
def test_fp32_tensor_core_products(nx, ny, p, nrhs):
    # FP32 sweep products on the tensor cores (three bf16 pieces per entry) and on the FP32
    # FFMA pipe: both refined solutions within 1e-8 of the oracle, and of each other; nrhs
    # 100 spans two 64-column units per operator block, 9 leaves most of one unused
    from paper_1612_02736_gb300 import Solver
    case = make_case(nx, ny, p, nrhs=nrhs)
    (uc, ug), _ = oracle_solve(case)
    out = {}
    for mode in ("tensor", "simt"):
        s = Solver(gpu_tree(case), to_dev(case["coeffs"]), p, precision="mixed", fp32_gemm=mode)
        for _ in range(2):  # the second solve runs the calibrated schedule
            u, ugg = s.solve(to_dev(case["f"]), to_dev(case["g"]), return_gauss=True)
            assert rel_linf(u.cpu().numpy(), uc) < 1e-8, (mode, rel_linf(u.cpu().numpy(), uc))
            assert rel_linf(ugg.cpu().numpy(), ug) < 1e-8
        out[mode] = u.cpu().numpy()
    assert rel_linf(out["tensor"], out["simt"]) < 1e-8
