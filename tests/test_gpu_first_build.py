"""A build whose kernels need more than the default 48 KB of shared memory once their
static shared memory is counted, as the first build of a fresh process (p = 20: the leaf
panel takes 45 KB of dynamic shared memory): it must build and solve, and agree with the
oracle.  Run in a child process so that no earlier launch has raised any limit."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np, torch
from paper_1612_02736_gb300 import Solver
from tests.gpu_common import gpu_tree, make_case, oracle_solve, to_dev
from tests.helpers import rel_linf
for prec, tol in (("fp64", 1e-10), ("mixed", 1e-8)):
    case = make_case(2, 2, 20, nrhs=3)
    (uc, _), _ = oracle_solve(case)
    u = Solver(gpu_tree(case), to_dev(case["coeffs"]), 20, precision=prec).solve(to_dev(case["f"]), to_dev(case["g"]))
    err = rel_linf(u.cpu().numpy(), uc)
    assert err < tol, (prec, err)
print("ok")
""".replace("ROOT", repr(ROOT))


def test_first_build_of_a_process_at_p20():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
