"""Failure paths of the build and solve, made on the host or by the inputs (no GPU fault):
non-elliptic or non-finite coefficient fields, a singular leaf, an allocator that fails on
its k-th request, and a bounded device wait that runs out (a barrier nothing arrives at).
Each returns its status code, releases what it allocated, and leaves the library usable for
the next call."""
import ctypes as C

import numpy as np
import pytest

from oracle import leaf as lfm, spectral as sp
from tests.gpu_common import gpu_tree, make_case, oracle_solve, to_dev
from tests.helpers import rel_linf

pytestmark = pytest.mark.gpu

HPS_ERR_INVALID_ARG, HPS_ERR_NOT_ELLIPTIC, HPS_ERR_SINGULAR, HPS_ERR_OOM, HPS_ERR_TIMEOUT = 1, 2, 3, 4, 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


def _solver_error(coeffs, p, nx=2, ny=2, **kw):
    from paper_1612_02736_gb300 import HPSError, Solver, Tree
    t = Tree.uniform(0.0, 0.0, 1.0, 1.0, nx, ny)
    with pytest.raises(HPSError) as ei:
        Solver(t, coeffs, p, **kw)
    return ei.value


def _still_usable():
    # a small build and solve right after a failure match the oracle
    from paper_1612_02736_gb300 import Solver
    case = make_case(2, 2, 8)
    (uc, _), _ = oracle_solve(case)
    u = Solver(gpu_tree(case), to_dev(case["coeffs"]), 8).solve(to_dev(case["f"]), to_dev(case["g"]))
    assert rel_linf(u.cpu().numpy(), uc) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_elliptic_coefficients(precision):
    case = make_case(2, 2, 8)
    c = case["coeffs"].copy()
    node = 3 * 8 + 4                       # an interior node (ix = 4, iy = 3) of leaf 2
    c[1, 2, node] = 2.0 * np.sqrt(c[0, 2, node] * c[2, 2, node])   # c12^2 > c11 c22
    e = _solver_error(to_dev(c), 8, precision=precision)
    assert e.code == HPS_ERR_NOT_ELLIPTIC and "leaf 2" in str(e)
    c = case["coeffs"].copy()
    c[0, 1, node] = -1.0                   # c11 < 0 in leaf 1
    e = _solver_error(to_dev(c), 8, precision=precision)
    assert e.code == HPS_ERR_NOT_ELLIPTIC and "leaf 1" in str(e)
    zero = np.zeros_like(case["coeffs"])
    assert _solver_error(to_dev(zero), 8, precision=precision).code == HPS_ERR_NOT_ELLIPTIC
    _still_usable()


def test_non_finite_coefficients():
    from paper_1612_02736_gb300 import Solver
    case = make_case(2, 2, 8)
    for bad in (np.nan, np.inf):
        c = case["coeffs"].copy()
        c[5, 3, 2 * 8 + 5] = bad           # interior node of leaf 3, field c
        e = _solver_error(to_dev(c), 8)
        assert e.code == HPS_ERR_INVALID_ARG and "leaf 3" in str(e)
    # exterior coefficient values are never used: a NaN there is accepted
    c = case["coeffs"].copy()
    c[:, 0, 0] = np.nan
    (uc, _), _ = oracle_solve(case)
    u = Solver(gpu_tree(case), to_dev(c), 8).solve(to_dev(case["f"]), to_dev(case["g"]))
    assert rel_linf(u.cpu().numpy(), uc) < 1e-10
    _still_usable()


def test_singular_leaf():
    # -Laplace(u) - lam u with lam an eigenvalue of the leaf's interior block (p = 4): the
    # coefficients are elliptic, the leaf system is singular and its elimination breaks down
    import torch
    p, h = 4, 0.5
    ones = np.ones(p * p)
    A = lfm.leaf_A([ones, 0 * ones, ones, 0 * ones, 0 * ones, 0 * ones], p, h, h)
    _, ci, _ = sp.leaf_index_sets(p)
    lam = np.linalg.eigvals(A[np.ix_(ci, ci)])
    lam = float(np.min(np.real(lam[np.abs(np.imag(lam)) < 1e-12])))
    c = torch.zeros((6, 4, p * p), dtype=torch.float64, device="cuda")
    c[0] = 1.0
    c[2] = 1.0
    c[5] = -lam
    e = _solver_error(c, p)
    assert e.code == HPS_ERR_SINGULAR and "box" in str(e)
    _still_usable()


class _CountingAllocator:
    """hps_allocator over torch's caching allocator that fails its k-th request and counts
    live blocks."""

    def __init__(self, fail_at):
        import torch
        from paper_1612_02736_gb300 import _native as N
        self.fail_at, self.calls, self.live = fail_at, 0, set()

        def alloc(nbytes, ctx, stream):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            self.live.add(ptr)
            return ptr

        def free(ptr, ctx, stream):
            if ptr:
                self.live.discard(ptr)
                torch.cuda.caching_allocator_delete(int(ptr))

        self._a, self._f = N.ALLOC_FN(alloc), N.FREE_FN(free)
        self.struct = N.hps_allocator(self._a, self._f, None)


def test_allocation_failures_release_everything():
    # the build fails at every one of its allocations in turn: OOM each time, no block left
    # behind; then a build succeeds and a solve whose workspace allocation fails reports OOM
    # and leaves the handle usable
    import torch
    from paper_1612_02736_gb300 import _native as N
    lib = N.load()
    case = make_case(2, 2, 8, nrhs=2)
    (uc, _), _ = oracle_solve(case)
    tree = C.c_void_p()
    assert lib.hps_tree_uniform(0.0, 0.0, 1.0, 1.0, 2, 2, C.byref(tree)) == 0
    coeffs = to_dev(case["coeffs"])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = C.c_void_p()
    k = 1
    while True:
        al = _CountingAllocator(k)
        rc = lib.hps_build(tree, C.c_void_p(coeffs.data_ptr()), 8, None, C.byref(al.struct), stream, C.byref(h))
        torch.cuda.synchronize()
        if rc == 0:
            break
        assert rc == HPS_ERR_OOM, lib.hps_last_error()
        assert not h.value and not al.live, (k, len(al.live))
        k += 1
        assert k < 500
    assert k > 5   # the build allocates many blocks: each failure point was exercised
    f, g = to_dev(case["f"]), to_dev(case["g"])
    u = torch.empty_like(g)
    al.fail_at = al.calls + 1                  # the solve's first workspace allocation fails
    rc = lib.hps_solve(h, C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), 2, C.c_void_p(u.data_ptr()), stream)
    assert rc == HPS_ERR_OOM
    rc = lib.hps_solve(h, C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), 2, C.c_void_p(u.data_ptr()), stream)
    assert rc == 0, lib.hps_last_error()
    torch.cuda.synchronize()
    assert rel_linf(u.cpu().numpy(), uc) < 1e-10
    assert lib.hps_destroy(h) == 0
    assert not al.live
    lib.hps_tree_destroy(tree)


def test_bounded_wait_runs_out():
    # the bounded wait of the tensor-core kernels on a barrier that nothing arrives at: it
    # gives up after its poll limit, raises the abort flag that stops the other role, and
    # the call reports TIMEOUT; the device is usable afterwards
    import torch
    from paper_1612_02736_gb300 import _native as N
    lib = N.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for polls in (1, 1000, 100000):
        rc = lib.hps_selftest_wait_timeout(polls, stream)
        assert rc == HPS_ERR_TIMEOUT, (polls, rc, lib.hps_last_error())
    _still_usable()
