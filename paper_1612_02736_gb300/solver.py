"""Python front end of the GB300 HPS solver: thin wrappers over the C ABI.

PyTorch provides device memory (the library allocates through torch's caching allocator)
and streams (every call runs on torch's current CUDA stream).  All arithmetic happens in
``libhps_gb300.so``.
"""
import ctypes as C

import numpy as np
import torch

from . import _native as N


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class _TorchAllocator:
    """hps_allocator bound to torch's CUDA caching allocator."""

    def __init__(self):
        def alloc(nbytes, ctx, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            except Exception:  # OOM -> NULL, reported as HPS_ERR_OOM by the library
                return None

        def free(ptr, ctx, stream):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._a = N.ALLOC_FN(alloc)
        self._f = N.FREE_FN(free)
        self.struct = N.hps_allocator(self._a, self._f, None)


_ALLOCATOR = None


def _allocator():
    global _ALLOCATOR
    if _ALLOCATOR is None:
        _ALLOCATOR = _TorchAllocator()
    return _ALLOCATOR


class Tree:
    """A box tree (Sec. 2).  Leaves are numbered j * nx + i."""

    def __init__(self, ptr, nx, ny, rect):
        self._ptr = ptr
        self.nx, self.ny, self.rect = nx, ny, rect

    @classmethod
    def uniform(cls, x0, y0, x1, y1, nx, ny):
        lib = N.load()
        out = C.c_void_p()
        N.check(lib.hps_tree_uniform(x0, y0, x1, y1, nx, ny, C.byref(out)))
        return cls(out, nx, ny, (x0, y0, x1, y1))

    @classmethod
    def mask(cls, x0, y0, h, mask):
        """Union of squares of side h: mask[j][i] != 0 keeps the square (i, j)."""
        lib = N.load()
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        ny, nx = m.shape
        out = C.c_void_p()
        N.check(lib.hps_tree_mask(x0, y0, h, nx, ny, m.ctypes.data_as(C.c_void_p), C.byref(out)))
        return cls(out, nx, ny, (x0, y0, x0 + nx * h, y0 + ny * h))

    @classmethod
    def l_shape(cls, n):
        """[-1,1]^2 minus [0,1] x [-1,0] on a 2n x 2n grid of squares."""
        m = np.ones((2 * n, 2 * n), dtype=np.uint8)
        m[:n, n:] = 0
        return cls.mask(-1.0, -1.0, 1.0 / n, m)

    def refine(self, points, levels):
        """A new tree refined `levels` times toward the points (Sec. 6.1)."""
        lib = N.load()
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 2))
        out = C.c_void_p()
        N.check(lib.hps_tree_refine(self._ptr, pts.ctypes.data_as(C.c_void_p), len(pts), levels, C.byref(out)))
        return Tree(out, self.nx, self.ny, self.rect)

    def info(self, q):
        vals = [C.c_int() for _ in range(5)]
        N.check(N.load().hps_tree_info(self._ptr, q, *[C.byref(v) for v in vals]))
        keys = ("n_leaves", "n_boxes", "n_levels", "n_gauss", "n_boundary")
        return {k: v.value for k, v in zip(keys, vals)}

    def nodes(self, p, q, which):
        """Node coordinates as a (count, 2) float64 array.  which: 'cheb', 'boundary', 'gauss'."""
        code = {"cheb": N.HPS_NODES_CHEB_LEAF, "boundary": N.HPS_NODES_GAUSS_BOUNDARY,
                "gauss": N.HPS_NODES_GAUSS_ALL}[which]
        lib = N.load()
        cnt = C.c_int64()
        N.check(lib.hps_nodes(self._ptr, p, q, code, None, C.byref(cnt)))
        out = np.zeros((cnt.value, 2), dtype=np.float64)
        N.check(lib.hps_nodes(self._ptr, p, q, code, out.ctypes.data_as(C.c_void_p), C.byref(cnt)))
        return out

    def close(self):
        if self._ptr:
            N.load().hps_tree_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_rhs(x, rows, name):
    if x.dim() == 1:
        x = x.unsqueeze(-1)
    if x.shape[0] != rows:
        raise ValueError("%s has %d rows, expected %d" % (name, x.shape[0], rows))
    return x


class Solver:
    """Build stage (Algorithm 1) on construction; solve (Algorithm 2) and adjoint on call.

    coeffs: CUDA float64 tensor (6, n_leaf, p*p) with c11, c12, c22, c1, c2, c at every leaf
    Chebyshev node.  precision: 'fp64' or 'mixed' (FP32 sweeps + FP64 iterative refinement).
    autotune: time the candidate tile configurations of each new launch shape once and keep
    the fastest (autotune_cache: a text file that keeps the choices across processes).
    shared_leaf: "auto" stores one leaf's operators for all leaves when every leaf has the
    same size and interior coefficients (constant-coefficient problems); True requires it,
    False never shares.
    bc_we ("dirichlet" | "periodic") and bc_sn ("dirichlet" | "neumann"): boundary kinds of
    the west/east and south/north sides of a rectangular domain (Sec. 7.6); f then holds
    Dirichlet values, or du/dy on Neumann sides, and is ignored on periodic sides.
    fp64_gemm: "tensor" runs the FP64 solve and adjoint products on the tensor cores by exact
    digit slicing where they apply (inner dimension <= 448, nrhs >= 8), "simt" on the FP64
    FFMA pipe throughout.  fp32_gemm: the FP32 sweep products of the mixed path with more
    than 8 right-hand sides on the tensor cores ("tensor", three bf16 pieces per entry) or
    on the FP32 FFMA pipe ("simt").
    """

    def __init__(self, tree, coeffs, p, precision="fp64", q=None, ir_tol=None, ir_max_iter=None,
                 fp64_top_levels=None, store_leaf_ops=True, use_graphs=True, autotune=False,
                 autotune_cache=None, shared_leaf="auto", bc_we="dirichlet", bc_sn="dirichlet",
                 fp64_gemm="tensor", fp32_gemm="tensor", allocator="torch"):
        lib = N.load()
        if not (coeffs.is_cuda and coeffs.dtype == torch.float64 and coeffs.is_contiguous()):
            raise ValueError("coeffs must be a contiguous CUDA float64 tensor")
        opts = N.hps_opts()
        lib.hps_opts_default(C.byref(opts))
        opts.precision = {"fp64": N.HPS_FP64, "mixed": N.HPS_MIXED}[precision]
        if q is not None:
            opts.q = q
        if ir_tol is not None:
            opts.ir_tol = ir_tol
        if ir_max_iter is not None:
            opts.ir_max_iter = ir_max_iter
        if fp64_top_levels is not None:
            opts.fp64_top_levels = fp64_top_levels
        opts.store_leaf_ops = 1 if store_leaf_ops else 0
        opts.use_graphs = 1 if use_graphs else 0
        opts.autotune = 1 if autotune else 0
        self._tune_path = None if autotune_cache is None else str(autotune_cache).encode()
        opts.autotune_cache = self._tune_path
        opts.shared_leaf = {"auto": -1, False: 0, True: 1}[shared_leaf]
        opts.bc_we = {"dirichlet": N.HPS_BC_DIRICHLET, "periodic": N.HPS_BC_PERIODIC}[bc_we]
        opts.bc_sn = {"dirichlet": N.HPS_BC_DIRICHLET, "neumann": N.HPS_BC_NEUMANN}[bc_sn]
        opts.fp64_gemm = {"tensor": N.HPS_GEMM_TENSOR, "simt": N.HPS_GEMM_SIMT}[fp64_gemm]
        opts.fp32_gemm = {"tensor": N.HPS_GEMM_TENSOR, "simt": N.HPS_GEMM_SIMT}[fp32_gemm]
        self.tree, self.p, self.precision = tree, p, precision
        self._alloc = _allocator() if allocator == "torch" else None
        out = C.c_void_p()
        N.check(lib.hps_build(tree._ptr, _ptr(coeffs), p, C.byref(opts),
                              C.byref(self._alloc.struct) if self._alloc else None, _stream(), C.byref(out)))
        self._h = out
        vals = [C.c_int() for _ in range(5)]
        ob = C.c_int64()
        N.check(lib.hps_handle_info(self._h, *[C.byref(v) for v in vals], C.byref(ob)))
        self.n_leaf, _, self.q, self.n_gauss, self.n_bdry = [v.value for v in vals]
        self.operator_bytes = ob.value
        self.last_iters = 0

    def solve(self, f, g, rho=None, return_gauss=False):
        """u at every leaf Chebyshev node; f (n_bdry[, nrhs]), g (n_leaf, p*p[, nrhs])."""
        squeeze = g.dim() == 2
        g = g.unsqueeze(-1) if squeeze else g
        nrhs = g.shape[-1]
        f = _as_rhs(f, self.n_bdry, "f").contiguous()
        g = g.contiguous()
        for t in (f, g):
            if not (t.is_cuda and t.dtype == torch.float64):
                raise ValueError("f and g must be CUDA float64 tensors")
        if f.shape[-1] != nrhs:
            raise ValueError("f and g disagree on nrhs")
        u = torch.empty_like(g)
        ug = torch.empty((self.n_gauss, nrhs), dtype=torch.float64, device=g.device) if return_gauss else None
        if rho is not None:
            rho = _as_rhs(rho, self.n_gauss, "rho").contiguous()
        it = C.c_int()
        N.check(N.load().hps_solve_ext(self._h, _ptr(f), _ptr(g), _ptr(rho), nrhs, _ptr(u), _ptr(ug),
                                       C.byref(it), _stream()))
        self.last_iters = it.value
        if squeeze:
            u = u.squeeze(-1)
            if ug is not None:
                ug = ug.squeeze(-1)
        return (u, ug) if return_gauss else u

    def apply(self, coeffs, u, alpha=0.0, beta=1.0):
        """alpha u + beta A u at every leaf's interior Chebyshev nodes (0 at the exterior
        ones), A the collocation operator for the coefficient fields coeffs (6, n_leaf,
        p*p); u is (n_leaf, p*p[, nrhs])."""
        squeeze = u.dim() == 2
        uu = (u.unsqueeze(-1) if squeeze else u).contiguous()
        if not (coeffs.is_cuda and coeffs.dtype == torch.float64 and coeffs.is_contiguous()):
            raise ValueError("coeffs must be a contiguous CUDA float64 tensor")
        out = torch.empty_like(uu)
        N.check(N.load().hps_apply(self._h, _ptr(coeffs), _ptr(uu), uu.shape[-1], float(alpha), float(beta),
                                   _ptr(out), _stream()))
        return out.squeeze(-1) if squeeze else out

    def adjoint(self, dJdu, u=None, want_coeffs=True):
        """(dJ/df, dJ/dg, dJ/dcoeffs) for the gradient dJdu of the solution; dJ/dcoeffs
        needs the forward solution u and is summed over right-hand sides."""
        squeeze = dJdu.dim() == 2
        ub = (dJdu.unsqueeze(-1) if squeeze else dJdu).contiguous()
        nrhs = ub.shape[-1]
        fb = torch.empty((self.n_bdry, nrhs), dtype=torch.float64, device=ub.device)
        gb = torch.empty_like(ub)
        cb = None
        if want_coeffs:
            if u is None:
                raise ValueError("coefficient gradients need the forward solution u")
            u = (u.unsqueeze(-1) if u.dim() == 2 else u).contiguous()
            cb = torch.empty((6, self.n_leaf, self.p * self.p), dtype=torch.float64, device=ub.device)
        N.check(N.load().hps_adjoint(self._h, _ptr(ub), nrhs, _ptr(u) if want_coeffs else None, _ptr(fb),
                                     _ptr(gb), _ptr(cb), _stream()))
        if squeeze:
            fb, gb = fb.squeeze(-1), gb.squeeze(-1)
        return fb, gb, cb

    def close(self):
        if getattr(self, "_h", None):
            N.load().hps_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HPSFunction(torch.autograd.Function):
    """u = Sol(coeffs, f, g) with a hand-written backward: one transposed sweep through the
    stored FP64 factorization (hps_adjoint) gives dJ/df, dJ/dg and dJ/dcoeffs."""

    @staticmethod
    def forward(ctx, coeffs, f, g, tree, p, store_leaf_ops=True):
        solver = Solver(tree, coeffs.detach().contiguous(), p, precision="fp64", store_leaf_ops=store_leaf_ops)
        u = solver.solve(f.detach(), g.detach())
        ctx.solver = solver
        ctx.save_for_backward(u)
        ctx.f_shape, ctx.g_shape = f.shape, g.shape
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        fb, gb, cb = ctx.solver.adjoint(gu.contiguous(), u=u, want_coeffs=ctx.needs_input_grad[0])
        ctx.solver.close()
        return (cb if ctx.needs_input_grad[0] else None,
                fb.reshape(ctx.f_shape) if ctx.needs_input_grad[1] else None,
                gb.reshape(ctx.g_shape) if ctx.needs_input_grad[2] else None, None, None, None)
