"""The tile autotuner: builds and solves with autotuning match the oracle, and tuned
choices are stable within a process and written to the cache file."""
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


@pytest.mark.parametrize("precision,fp32_gemm", [("fp64", "tensor"), ("mixed", "tensor"), ("mixed", "simt")])
def test_autotuned_build_and_solve_match_oracle(precision, fp32_gemm, tmp_path):
    import torch
    from paper_1612_02736_gb300 import Solver
    cache = tmp_path / "tune.txt"
    case = make_case(8, 8, 12, nrhs=40)
    (uc, _), _ = oracle_solve(case)
    t = gpu_tree(case)
    f, g = to_dev(case["f"]), to_dev(case["g"])
    kw = {"fp32_gemm": fp32_gemm}
    s1 = Solver(t, to_dev(case["coeffs"]), 12, precision, autotune=True, autotune_cache=cache, **kw)
    u1 = s1.solve(f, g)
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert rel_linf(u1.cpu().numpy(), uc) < tol
    lines = cache.read_text().splitlines()
    assert any(l.startswith("gj_cfg leaf") for l in lines)
    assert any(l.startswith("gj_cfg merge") for l in lines)
    # right-hand-side tiles are tuned for the SIMT products only: the FP32 sweeps of the
    # mixed path when they run on the FP32 pipe; the FP64 products of this problem (inner
    # dimensions <= 448) and the FP32 ones by default run on the tensor cores, which have no
    # such tile
    tuned_f32 = any(l.startswith("gemm_bn leaf_down f32") for l in lines)
    assert tuned_f32 == (precision == "mixed" and fp32_gemm == "simt")
    assert not any(l.startswith("gemm_bn") and " f64 " in l for l in lines)
    for l in lines:
        # panel width (+ 100 for the tensor-core FP64 update) or right-hand-side tile
        assert int(l.rsplit(" ", 1)[1]) in (4, 8, 16, 32, 64, 104, 108, 116)
    # the same shapes again: choices come from memory, results are reproduced bit for bit
    s2 = Solver(t, to_dev(case["coeffs"]), 12, precision, autotune=True, autotune_cache=cache, **kw)
    u2 = s2.solve(f, g)
    assert torch.equal(u1, u2)
    assert cache.read_text().splitlines() == lines
    # against the fixed rules: only the panel widths' rounding differs
    s3 = Solver(t, to_dev(case["coeffs"]), 12, precision, **kw)
    assert rel_linf(s3.solve(f, g).cpu().numpy(), u1.cpu().numpy()) < (1e-12 if precision == "fp64" else 1e-8)
