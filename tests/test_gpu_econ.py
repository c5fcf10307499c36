"""Leaf recomputation ("econ", store_leaf_ops = 0; the storage-efficient variant of the
Sec. 5.4 remark): the solve and the adjoint rebuild F, S, H chunk by chunk and must give
the oracle's results."""
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


@pytest.mark.parametrize("nx,ny,p,nrhs", [(4, 4, 10, 1), (8, 8, 16, 8), (5, 3, 9, 3)])
def test_econ_solve_and_adjoint_match_oracle(nx, ny, p, nrhs):
    from paper_1612_02736_gb300 import Solver
    case = make_case(nx, ny, p, nrhs=nrhs)
    (uc, _), ops = oracle_solve(case)
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), p, store_leaf_ops=False)
    u = s.solve(to_dev(case["f"]), to_dev(case["g"]))
    assert rel_linf(u.cpu().numpy(), uc) < 1e-10
    ubar = np.random.default_rng(5).standard_normal(uc.shape)
    fb, gb, _ = hps.adjoint(case["tree"], ops, p, ubar)
    cg = hps.coeff_gradients(case["tree"], p, uc, gb)
    fbg, gbg, cgg = s.adjoint(to_dev(ubar), u=u)
    assert rel_linf(fbg.cpu().numpy(), fb) < 1e-9
    assert rel_linf(gbg.cpu().numpy(), gb) < 1e-9
    assert rel_linf(cgg.cpu().numpy(), cg) < 1e-9


def test_econ_equals_stored_at_full_size():
    # 64 x 64 leaves, p = 16: several recomputation chunks; same kernels, same results.
    from paper_1612_02736_gb300 import Solver
    import torch
    case = make_case(64, 64, 16, nrhs=2)
    f, g = to_dev(case["f"]), to_dev(case["g"])
    a = Solver(gpu_tree(case), to_dev(case["coeffs"]), 16)
    b = Solver(gpu_tree(case), to_dev(case["coeffs"]), 16, store_leaf_ops=False)
    assert b.operator_bytes < 0.5 * a.operator_bytes
    ua, ub = a.solve(f, g), b.solve(f, g)
    assert ((ua - ub).abs().max() / ua.abs().max()).item() < 1e-12
    ga = a.adjoint(ua, u=ua)[1]
    gb = b.adjoint(ub, u=ub)[1]
    assert ((ga - gb).abs().max() / ga.abs().max()).item() < 1e-12
    torch.cuda.synchronize()
