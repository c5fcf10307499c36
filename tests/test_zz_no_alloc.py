"""hps_solve_noalloc: the solve for callers that cannot let it allocate device memory (a
framework that has reserved nearly all of it, a running time-stepping loop).  Checked
through the C ABI against hps_solve on the same handle, on two calls in a row with
different data, plus its size limit; also with the tensor-core products (8 and more
right-hand sides, before and after hps_solve has cached the operator digits), on a handle
that recomputes its leaf operators, and on a locally refined tree.  Kept in a file of its
own that is collected last."""
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


def _handle(lib, case, precision=0, store_leaf_ops=1, tree=None):
    from paper_1612_02736_gb300 import _native
    own = tree is None
    if own:
        tree = C.c_void_p()
        assert lib.hps_tree_uniform(*case["rect"], case["nx"], case["ny"], C.byref(tree)) == 0
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.precision = precision
    opts.store_leaf_ops = store_leaf_ops
    coeffs = _dev(case["coeffs"])
    h = C.c_void_p()
    rc = lib.hps_build(tree, _ptr(coeffs), case["p"], C.byref(opts), None, None, C.byref(h))
    assert rc == 0, lib.hps_last_error()
    if own:
        lib.hps_tree_destroy(tree)
    return h


def _compare(lib, h, f_h, g_h, nrhs, noalloc_first=False):
    """hps_solve_noalloc against hps_solve on the same inputs; returns the relative error."""
    import torch
    f, g = _dev(f_h), _dev(g_h)
    ref = torch.empty_like(g)
    out = torch.full_like(g, np.nan)
    calls = [(lib.hps_solve_noalloc, out), (lib.hps_solve, ref)]
    if not noalloc_first:
        calls.reverse()
    for fn, dst in calls:
        assert fn(h, _ptr(f), _ptr(g), nrhs, _ptr(dst), None) == 0, lib.hps_last_error()
    torch.cuda.synchronize()
    return ((out - ref).abs().max() / ref.abs().max()).item()


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


@pytest.mark.parametrize("nrhs", [8, 16])
def test_noalloc_tensor_core_products(lib, nrhs):
    # from 8 right-hand sides the FP64 products run on the tensor cores, whose exponents
    # then come from the fixed array too: on a fresh handle (no operator digits cached yet)
    # and after hps_solve has cached them (from its second call on)
    case = make_case(16, 16, 12, nrhs=nrhs)
    h = _handle(lib, case)
    f, g = case["f"], case["g"]
    assert _compare(lib, h, f, g, nrhs, noalloc_first=True) < 1e-10
    for k in range(3):
        assert _compare(lib, h, (1.0 + k) * f, g - k, nrhs) < 1e-10
    lib.hps_destroy(h)


@pytest.mark.parametrize("nrhs", [3, 8])
def test_noalloc_recomputed_leaf_operators(lib, nrhs):
    # store_leaf_ops = 0: the leaf operators are rebuilt chunk by chunk inside the call,
    # in buffers the handle allocated at build time
    case = make_case(16, 16, 12, nrhs=nrhs)
    h = _handle(lib, case, store_leaf_ops=0)
    for k in range(2):
        assert _compare(lib, h, case["f"] * (k + 1), case["g"] + k, nrhs) < 1e-10
    lib.hps_destroy(h)


def test_noalloc_refined_tree(lib):
    # a locally refined tree (coarse-fine interpolation items in the sweep)
    base = C.c_void_p()
    assert lib.hps_tree_uniform(0.0, 0.0, 1.0, 1.0, 4, 4, C.byref(base)) == 0
    pts = np.array([0.3, 0.7], dtype=np.float64)
    tree = C.c_void_p()
    assert lib.hps_tree_refine(base, pts.ctypes.data_as(C.c_void_p), 1, 2, C.byref(tree)) == 0
    p, nrhs = 10, 2
    vals = [C.c_int() for _ in range(5)]
    assert lib.hps_tree_info(tree, p - 1, *[C.byref(v) for v in vals]) == 0
    n_leaf, n_bdry = vals[0].value, vals[4].value
    rng = np.random.default_rng(5)
    coeffs = np.zeros((6, n_leaf, p * p))
    coeffs[0] = 1.0 + 0.1 * rng.random((n_leaf, p * p))
    coeffs[2] = 1.0 + 0.1 * rng.random((n_leaf, p * p))
    coeffs[5] = rng.random((n_leaf, p * p))
    case = {"coeffs": coeffs, "p": p}
    h = _handle(lib, case, tree=tree)
    for k in range(2):
        f = rng.standard_normal((n_bdry, nrhs))
        g = rng.standard_normal((n_leaf, p * p, nrhs))
        assert _compare(lib, h, f, g, nrhs, noalloc_first=(k == 0)) < 1e-10
    lib.hps_destroy(h)
    lib.hps_tree_destroy(tree)
    lib.hps_tree_destroy(base)
