"""CPU checks of the native library: it loads, exports every symbol of include/hps.h, and
its host logic (tree, node numbering, node coordinates, argument checks) agrees with the
oracle.  No kernel is launched here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import spectral as sp
from oracle import tree as tr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_02736_gb300 import build, _native
    build.build()
    return _native.load()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "hps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hps_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_1612_02736_gb300 import _native
    syms = header_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
        assert s in _native.SIGNATURES, s


def _tree(lib, nx, ny, rect=(0.0, 0.0, 1.0, 1.0)):
    out = C.c_void_p()
    assert lib.hps_tree_uniform(*rect, nx, ny, C.byref(out)) == 0
    return out


@pytest.mark.parametrize("nx,ny,q", [(1, 1, 5), (2, 2, 7), (4, 4, 15), (8, 4, 9), (64, 64, 15)])
def test_tree_counts_match_oracle(lib, nx, ny, q):
    t = _tree(lib, nx, ny)
    vals = [C.c_int() for _ in range(5)]
    assert lib.hps_tree_info(t, q, *[C.byref(v) for v in vals]) == 0
    n_leaves, n_boxes, n_levels, n_gauss, n_bdry = [v.value for v in vals]
    assert n_leaves == nx * ny and n_boxes == 2 * nx * ny - 1
    o = tr.uniform_tree(0, 0, 1, 1, nx, ny, q)
    assert n_gauss == o.n_gauss and n_bdry == len(o.boundary)
    lib.hps_tree_destroy(t)


@pytest.mark.parametrize("nx,ny,p", [(2, 2, 8), (4, 2, 16)])
def test_node_coordinates_match_oracle(lib, nx, ny, p):
    q = p - 1
    rect = (0.25, -0.5, 1.25, 0.5)
    t = _tree(lib, nx, ny, rect)
    o = tr.uniform_tree(*rect, nx, ny, q)

    def get(which):
        cnt = C.c_int64()
        assert lib.hps_nodes(t, p, q, which, None, C.byref(cnt)) == 0
        xy = np.zeros((cnt.value, 2))
        assert lib.hps_nodes(t, p, q, which, xy.ctypes.data_as(C.c_void_p), C.byref(cnt)) == 0
        return xy

    cheb = get(0)
    X, Y = [], []
    for lf in range(o.n_leaves):
        x0, y0, x1, y1 = o.leaf_rect(lf)
        x, y = sp.leaf_cheb_points(x0, y0, x1 - x0, y1 - y0, p)
        X.append(x)
        Y.append(y)
    assert np.max(np.abs(cheb[:, 0] - np.concatenate(X))) < 1e-14
    assert np.max(np.abs(cheb[:, 1] - np.concatenate(Y))) < 1e-14
    gp = o.gauss_points()
    assert np.max(np.abs(get(2) - gp)) < 1e-14            # every Gaussian node by global id
    assert np.max(np.abs(get(1) - gp[o.boundary])) < 1e-14  # boundary order
    lib.hps_tree_destroy(t)


def test_invalid_arguments_report_errors(lib):
    out = C.c_void_p()
    assert lib.hps_tree_uniform(0.0, 0.0, 1.0, 1.0, 0, 3, C.byref(out)) == 1
    assert b"nx" in lib.hps_last_error()
    assert lib.hps_tree_uniform(1.0, 0.0, 0.0, 1.0, 2, 2, C.byref(out)) == 1
    t = _tree(lib, 2, 2)
    h = C.c_void_p()
    assert lib.hps_build(t, None, 8, None, None, None, C.byref(h)) == 1
    assert lib.hps_build(t, C.c_void_p(16), 3, None, None, None, C.byref(h)) == 1
    assert b"p must be" in lib.hps_last_error()
    assert lib.hps_solve(None, None, None, 1, None, None) == 1
    assert lib.hps_adjoint(None, None, 1, None, None, None, None, None) == 1
    cnt = C.c_int64()
    assert lib.hps_nodes(t, 8, 7, 9, None, C.byref(cnt)) == 1
    assert lib.hps_destroy(None) == 0
    lib.hps_tree_destroy(t)


def test_python_package_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1612_02736_gb300 import _native
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(ImportError):
        _native.load()


@pytest.mark.parametrize("nx,ny,p,prec,store", [(1, 1, 8, 0, 1), (2, 1, 6, 0, 1), (2, 2, 16, 1, 1), (4, 4, 12, 1, 1),
                                                (8, 4, 16, 0, 1), (64, 64, 16, 0, 1), (16, 16, 20, 1, 1),
                                                (8, 8, 16, 0, 0), (64, 64, 16, 0, 0), (3, 5, 9, 0, 0),
                                                (128, 128, 16, 0, 1), (32, 32, 30, 1, 1), (64, 64, 24, 0, 1)])
def test_plan_descriptors_stay_in_bounds(lib, nx, ny, p, prec, store):
    # Every kernel descriptor of the build, solve and adjoint plans is checked against the
    # size of the buffer it addresses, on the host, before any launch; the larger trees
    # include the blocked merge eliminations' product items and vector-digit groups (K up
    # to 960 in chunks of at most 448).
    from paper_1612_02736_gb300 import _native
    t = _tree(lib, nx, ny)
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.precision = prec
    opts.store_leaf_ops = store
    assert lib.hps_plan_check(t, p, C.byref(opts)) == 0, lib.hps_last_error()
    lib.hps_tree_destroy(t)


@pytest.mark.parametrize("nx,ny", [(3, 2), (3, 3), (5, 7), (13, 1)])
def test_plan_non_power_of_two_trees(lib, nx, ny):
    # uneven trees: leaves at several depths, merges of one level with different sizes
    t = _tree(lib, nx, ny)
    assert lib.hps_plan_check(t, 8, None) == 0, lib.hps_last_error()
    lib.hps_tree_destroy(t)


@pytest.mark.parametrize("nx,ny,p,prec", [(1, 1, 8, 0), (2, 2, 16, 1), (64, 64, 16, 0), (5, 3, 10, 0),
                                         (128, 128, 16, 1)])
def test_plan_shared_leaf_operators_stay_in_bounds(lib, nx, ny, p, prec):
    # one leaf's operators and T block shared by every leaf (constant coefficients)
    from paper_1612_02736_gb300 import _native
    t = _tree(lib, nx, ny)
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.precision = prec
    opts.shared_leaf = 1
    assert lib.hps_plan_check(t, p, C.byref(opts)) == 0, lib.hps_last_error()
    lib.hps_tree_destroy(t)


def test_plan_shared_leaf_needs_equal_leaves(lib):
    from paper_1612_02736_gb300 import _native
    t = _tree(lib, 2, 2)
    pts = (C.c_double * 2)(0.1, 0.1)
    r = C.c_void_p()
    assert lib.hps_tree_refine(t, pts, 1, 1, C.byref(r)) == 0, lib.hps_last_error()
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.shared_leaf = 1
    assert lib.hps_plan_check(r, 8, C.byref(opts)) == 1
    assert "one size" in lib.hps_last_error().decode()
    opts.shared_leaf = -1
    assert lib.hps_plan_check(r, 8, C.byref(opts)) == 0, lib.hps_last_error()
    lib.hps_tree_destroy(r)
    lib.hps_tree_destroy(t)


@pytest.mark.parametrize("bc", [(1, 2), (1, 0), (0, 2)])
@pytest.mark.parametrize("nx,ny,p", [(1, 1, 8), (2, 2, 8), (4, 2, 7), (3, 5, 9), (16, 16, 17), (64, 64, 16)])
def test_plan_root_conditions_stay_in_bounds(lib, bc, nx, ny, p):
    # periodic west/east and Neumann south/north sides: seam and flux tables, products
    from paper_1612_02736_gb300 import _native
    t = _tree(lib, nx, ny)
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.bc_we, opts.bc_sn = bc
    assert lib.hps_plan_check(t, p, C.byref(opts)) == 0, lib.hps_last_error()
    opts.precision = 1
    assert lib.hps_plan_check(t, p, C.byref(opts)) == 1      # FP64 only
    lib.hps_tree_destroy(t)


def test_plan_root_conditions_need_a_rectangle(lib):
    from paper_1612_02736_gb300 import _native
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.bc_sn = 2
    mask = (C.c_uint8 * 4)(1, 0, 1, 1)        # an L of three unit squares
    t = C.c_void_p()
    assert lib.hps_tree_mask(0.0, 0.0, 1.0, 2, 2, mask, C.byref(t)) == 0, lib.hps_last_error()
    assert lib.hps_plan_check(t, 8, C.byref(opts)) == 1
    assert "rectangular" in lib.hps_last_error().decode()
    lib.hps_tree_destroy(t)
    # refined toward the west side only: facing west/east nodes no longer match
    u = _tree(lib, 2, 2)
    pts = (C.c_double * 2)(0.01, 0.5)
    r = C.c_void_p()
    assert lib.hps_tree_refine(u, pts, 1, 1, C.byref(r)) == 0, lib.hps_last_error()
    opts.bc_we = 1
    opts.bc_sn = 0
    assert lib.hps_plan_check(r, 8, C.byref(opts)) == 1
    assert "matching" in lib.hps_last_error().decode()
    opts.bc_we = 0
    opts.bc_sn = 2
    assert lib.hps_plan_check(r, 8, C.byref(opts)) == 0, lib.hps_last_error()
    lib.hps_tree_destroy(r)
    lib.hps_tree_destroy(u)


def test_plan_rejects_bad_options(lib):
    from paper_1612_02736_gb300 import _native
    t = _tree(lib, 2, 2)
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.precision = 7
    assert lib.hps_plan_check(t, 8, C.byref(opts)) == 1
    opts.precision = 0
    opts.q = 40
    assert lib.hps_plan_check(t, 8, C.byref(opts)) == 1
    lib.hps_opts_default(C.byref(opts))
    assert opts.fp64_gemm == _native.HPS_GEMM_TENSOR
    opts.fp64_gemm = _native.HPS_GEMM_SIMT
    assert lib.hps_plan_check(t, 8, C.byref(opts)) == 0
    opts.fp64_gemm = 5
    assert lib.hps_plan_check(t, 8, C.byref(opts)) == 1
    lib.hps_opts_default(C.byref(opts))
    assert opts.fp32_gemm == _native.HPS_GEMM_TENSOR
    opts.precision = _native.HPS_MIXED
    opts.fp32_gemm = _native.HPS_GEMM_SIMT
    assert lib.hps_plan_check(t, 8, C.byref(opts)) == 0
    opts.fp32_gemm = -1
    assert lib.hps_plan_check(t, 8, C.byref(opts)) == 1
    lib.hps_tree_destroy(t)


def _nodes(lib, t, p, q, which):
    cnt = C.c_int64()
    assert lib.hps_nodes(t, p, q, which, None, C.byref(cnt)) == 0
    xy = np.zeros((cnt.value, 2))
    assert lib.hps_nodes(t, p, q, which, xy.ctypes.data_as(C.c_void_p), C.byref(cnt)) == 0
    return xy


def _refined_pair(lib, kind, p):
    q = p - 1
    if kind == "uniform-refined":
        t = _tree(lib, 4, 4)
        o = tr.refine_tree(tr.uniform_tree(0, 0, 1, 1, 4, 4, q), [(0.37, 0.58), (0.9, 0.1)], 2)
        pts = np.array([[0.37, 0.58], [0.9, 0.1]])
        levels = 2
    else:
        m = np.ones((4, 4), dtype=np.uint8)
        m[:2, 2:] = 0
        t = C.c_void_p()
        assert lib.hps_tree_mask(-1.0, -1.0, 0.5, 4, 4, m.ctypes.data_as(C.c_void_p), C.byref(t)) == 0
        o = tr.refine_tree(tr.l_shape_tree(2, q), [(0.0, 0.0)], 3)
        pts = np.array([[0.0, 0.0]])
        levels = 3
    r = C.c_void_p()
    assert lib.hps_tree_refine(t, pts.ctypes.data_as(C.c_void_p), len(pts), levels, C.byref(r)) == 0
    lib.hps_tree_destroy(t)
    return r, o


@pytest.mark.parametrize("kind", ["uniform-refined", "l-shape-refined"])
def test_refined_and_mask_trees_match_oracle(lib, kind):
    p = 8
    q = p - 1
    r, o = _refined_pair(lib, kind, p)
    vals = [C.c_int() for _ in range(5)]
    assert lib.hps_tree_info(r, q, *[C.byref(v) for v in vals]) == 0
    assert vals[0].value == o.n_leaves and vals[3].value == o.n_gauss and vals[4].value == len(o.boundary)
    X, Y = [], []
    for lf in range(o.n_leaves):
        x0, y0, x1, y1 = o.leaf_rect(lf)
        x, y = sp.leaf_cheb_points(x0, y0, x1 - x0, y1 - y0, p)
        X.append(x)
        Y.append(y)
    cheb = _nodes(lib, r, p, q, 0)
    assert np.max(np.abs(cheb[:, 0] - np.concatenate(X))) < 1e-13
    assert np.max(np.abs(cheb[:, 1] - np.concatenate(Y))) < 1e-13
    gp = o.gauss_points()
    assert np.max(np.abs(_nodes(lib, r, p, q, 2) - gp)) < 1e-13
    assert np.max(np.abs(_nodes(lib, r, p, q, 1) - gp[o.boundary])) < 1e-13
    assert lib.hps_plan_check(r, p, None) == 0, lib.hps_last_error()
    from paper_1612_02736_gb300 import _native
    opts = _native.hps_opts()
    lib.hps_opts_default(C.byref(opts))
    opts.precision = 1
    assert lib.hps_plan_check(r, p, C.byref(opts)) == 1   # mixed needs matching interfaces
    lib.hps_tree_destroy(r)


def test_wait_selftest_rejects_bad_polls(lib):
    # argument checks happen before any device call
    assert lib.hps_selftest_wait_timeout(0, None) == 1
    assert lib.hps_selftest_wait_timeout((1 << 26) + 1, None) == 1
