"""hps_solve_noalloc: the solve for callers that cannot let it allocate device memory (a
framework that has reserved nearly all of it, a running time-stepping loop).  Checked
through the C ABI against hps_solve on the same handle, on two calls in a row with
different data, plus its size limit.  Kept in a file of its own that is collected last."""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_common import make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import _native, build
    build.build()
    return _native.load()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _handle(lib, case, precision=0):
    from paper_1612_02736_gb300 import _native
    tree = C.c_void_p()
    assert lib.hps_tree_uniform(*case["rect"], case["nx"], case["ny"], C.byref(tree)) == 0
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.precision = precision
    coeffs = _dev(case["coeffs"])
    h = C.c_void_p()
    rc = lib.hps_build(tree, _ptr(coeffs), case["p"], C.byref(opts), None, None, C.byref(h))
    assert rc == 0, lib.hps_last_error()
    lib.hps_tree_destroy(tree)
    return h


@pytest.mark.parametrize("nx,ny,p,nrhs", [(16, 16, 12, 3), (64, 64, 16, 1)])
def test_noalloc_matches_solve_on_two_calls(lib, nx, ny, p, nrhs):
    import torch
    case = make_case(nx, ny, p, nrhs=nrhs)
    h = _handle(lib, case)
    inputs = [(case["f"], case["g"]), (0.5 * case["f"] - 1.0, np.cos(case["g"]))]
    for f_h, g_h in inputs:  # two calls in a row, different data each time
        f, g = _dev(f_h), _dev(g_h)
        ref = torch.empty_like(g)
        out = torch.full_like(g, np.nan)
        assert lib.hps_solve(h, _ptr(f), _ptr(g), nrhs, _ptr(ref), None) == 0, lib.hps_last_error()
        assert lib.hps_solve_noalloc(h, _ptr(f), _ptr(g), nrhs, _ptr(out), None) == 0, lib.hps_last_error()
        torch.cuda.synchronize()
        err = ((out - ref).abs().max() / ref.abs().max()).item()
        assert err < 1e-10
    lib.hps_destroy(h)


def test_noalloc_rejects_oversized_calls_and_other_precisions(lib):
    import torch
    case = make_case(64, 64, 16, nrhs=1)
    h = _handle(lib, case)
    f = _dev(np.repeat(case["f"], 8, axis=1))
    g = _dev(np.repeat(case["g"], 8, axis=2))
    u = torch.empty_like(g)
    assert lib.hps_solve_noalloc(h, _ptr(f), _ptr(g), 8, _ptr(u), None) == 1
    assert b"scratch" in lib.hps_last_error()
    lib.hps_destroy(h)
    small = make_case(2, 2, 8)
    hm = _handle(lib, small, precision=1)
    f, g = _dev(small["f"]), _dev(small["g"])
    u = torch.empty_like(g)
    assert lib.hps_solve_noalloc(hm, _ptr(f), _ptr(g), 1, _ptr(u), None) == 8
    lib.hps_destroy(hm)
