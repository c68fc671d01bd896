"""Python front end of the xdcg library: Solver(K, Z).solve(f, tol) -> u, info.

Device memory and streams come from PyTorch; all arithmetic runs in the CUDA
library behind the C ABI (include/xdcg.h).
"""
import ctypes

import numpy as np
import torch

from . import _lib as L


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


class Elements:
    """Per-element data on the device for Solver.element_sensitivity: element
    e's local dofs dofs[dof_ptr[e]:dof_ptr[e+1]] (global dof, or -1 where
    eliminated) and its row-major unit-modulus stiffness at mats[mat_off[e]:]
    (layout of xdcg_element_sensitivity)."""

    def __init__(self, dof_ptr, dofs, mat_off, mats, device="cuda"):
        self.dof_ptr = torch.as_tensor(np.ascontiguousarray(dof_ptr, dtype=np.int64), device=device)
        self.dofs = torch.as_tensor(np.ascontiguousarray(dofs, dtype=np.int32), device=device)
        self.mat_off = torch.as_tensor(np.ascontiguousarray(mat_off, dtype=np.int64), device=device)
        self.mats = torch.as_tensor(np.ascontiguousarray(mats, dtype=np.float64), device=device)
        self.n_el = int(self.mat_off.numel())
        if self.dof_ptr.numel() != self.n_el + 1:
            raise ValueError("dof_ptr needs one entry more than mat_off")

    @classmethod
    def from_dict(cls, D, device="cuda"):
        return cls(D["dof_ptr"], D["dofs"], D["mat_off"], D["mats"], device)


class Pattern:
    """The stored block pattern of a node-blocked K on the device (dof_ptr,
    row_ptr, col, val_ptr), for Solver.stiffness_gradient."""

    def __init__(self, dof_ptr, row_ptr, col, val_ptr, device="cuda"):
        as_dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device=device)
        self.dof_ptr = as_dev(dof_ptr, np.int32)
        self.row_ptr = as_dev(row_ptr, np.int32)
        self.col = as_dev(col, np.int32)
        self.val_ptr = as_dev(val_ptr, np.int64)
        self.n_nodes = int(self.dof_ptr.numel()) - 1
        self.nval = int(self.val_ptr[-1].item())

    @classmethod
    def from_problem(cls, P, device="cuda"):
        return cls(P.dof_ptr, P.row_ptr, P.col, P.val_ptr, device)


class Solver:
    """Adapted deflated CG (A-DEF2 + node-block Jacobi) for one stiffness matrix.

    K: node-blocked CSR arrays (dof_ptr, row_ptr, col, val_ptr, val) in host memory;
    Z: box subdomains (sub_of_node, coords, hsign, centres).
    precision: "fp64" or "mixed" (FP32 PCG on the block-scaled system with FP64 residual replacement).
    jacobi: "block" (one block per node, the method's M) or "point" (diag K, the
    paper's comparison preconditioner).  record_history: keep ||r_i|| / ||f||
    per iteration of FP64 solves (history()).  coarse_fp64: mixed solves apply
    E^-1 in FP64 instead of its FP32 copy.  wait_s: limit of the SpMV's bounded
    waits on its own copies (xdcg_options.wait_s).  blocks: None (one block per
    node) or the block-Jacobi blocks as dof ranges, blocks[b] .. blocks[b+1]
    (whole nodes each; xdcg_blocks), e.g. one per subdomain of a problem
    numbered subdomain by subdomain.  z_cols, z_values: Z by value instead of
    from the geometry (xdcg_deflation's valued form: 6 or 12 columns per box,
    node I's b_I x z_cols[sub[I]] block row-major, nodes in order).  prev: a
    Solver of the same mesh for the previous crack front, whose unchanged
    parts are carried over (xdcg_setup_update).  graph: enqueue the solves'
    iterations as recorded CUDA graphs (xdcg_options.graph; same bits).
    spmv_shape: None, or (fp32_shape, fp64_shape) pinning the SpMV pipeline
    shapes (-1 keeps the default or the autotuner's pick).
    """

    def __init__(self, dof_ptr, row_ptr, col, val_ptr, val, sub_of_node, coords, hsign, centres,
                 precision="fp64", tol=1e-8, max_iter=10000, inner_tol=1e-3, max_outer=30,
                 time_spmv=False, enriched_modes=True, stream=None, jacobi="block",
                 record_history=False, max_batch=0, coarse_fp64=False, wait_s=2.0,
                 blocks=None, z_cols=None, z_values=None, prev=None, autotune=False,
                 graph=False, spmv_shape=None):
        lib = L.load()
        self._lib = lib
        self.ctx = ctypes.c_void_p()
        keep = [_host(dof_ptr, np.int32), _host(row_ptr, np.int32), _host(col, np.int32),
                _host(val_ptr, np.int64), _host(val, np.float64), _host(sub_of_node, np.int32),
                _host(coords, np.float64).reshape(-1), _host(hsign, np.int8),
                _host(centres, np.float64).reshape(-1)]
        n_nodes = keep[0].size - 1
        n_sub = keep[8].size // 3
        m = L.Matrix(n_nodes, keep[0].ctypes.data, keep[1].ctypes.data, keep[2].ctypes.data,
                     keep[3].ctypes.data, keep[4].ctypes.data, L.XDCG_HOST)
        z = L.Deflation(n_sub, keep[5].ctypes.data, keep[6].ctypes.data, keep[7].ctypes.data,
                        keep[8].ctypes.data, int(bool(enriched_modes)), L.XDCG_HOST, None, None)
        if z_values is not None:
            zc, zv = _host(z_cols, np.int32), _host(z_values, np.float64)
            keep += [zc, zv]
            z.sub_cols, z.values = zc.ctypes.data, zv.ctypes.data
        opt = L.Options()
        lib.xdcg_default_options(ctypes.byref(opt))
        opt.tol = tol
        opt.max_iter = max_iter
        opt.precision = L.XDCG_MIXED if precision == "mixed" else L.XDCG_FP64
        opt.inner_tol = inner_tol
        opt.max_outer = max_outer
        opt.time_spmv = 2 if time_spmv == "kernels" else int(bool(time_spmv))
        if jacobi not in ("block", "point"):
            raise ValueError("jacobi must be 'block' or 'point'")
        opt.jacobi = L.XDCG_POINT_JACOBI if jacobi == "point" else L.XDCG_BLOCK_JACOBI
        opt.record_history = int(bool(record_history))
        opt.max_batch = int(max_batch)
        opt.coarse_fp64 = int(bool(coarse_fp64))
        opt.wait_s = float(wait_s)
        opt.autotune = int(bool(autotune))
        opt.graph = int(bool(graph))
        if spmv_shape is not None:
            opt.spmv_shape_fp32, opt.spmv_shape_fp64 = (int(v) for v in spmv_shape)
        self.precision = precision
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        blk = None
        if blocks is not None:
            bp = _host(blocks, np.int32)
            keep.append(bp)
            blk = ctypes.byref(L.Blocks(bp.size - 1, bp.ctypes.data, L.XDCG_HOST))
        bad = ctypes.c_int32(-1)
        if prev is not None:
            # the next crack front of prev's mesh: unchanged node factors and an
            # unchanged E^-1 are carried over (xdcg_setup_update)
            st = lib.xdcg_setup_update(ctypes.byref(self.ctx), prev.ctx, ctypes.byref(m),
                                       ctypes.byref(z), blk, ctypes.byref(opt),
                                       ctypes.c_void_p(stream.cuda_stream), ctypes.byref(bad))
        else:
            st = lib.xdcg_setup(ctypes.byref(self.ctx), ctypes.byref(m), ctypes.byref(z), blk,
                                ctypes.byref(opt), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(bad))
        L.check(st, "xdcg_setup", bad.value)
        info = L.Info()
        L.check(lib.xdcg_get_info(self.ctx, ctypes.byref(info)), "xdcg_get_info")
        self.info = info.as_dict()
        self.n = int(info.n)
        self.k = int(info.k)

    @classmethod
    def from_problem(cls, P, **kw):
        return cls(P.dof_ptr, P.row_ptr, P.col, P.val_ptr, P.val, P.sub_of_node, P.coords,
                   P.hsign, P.centres, **kw)

    def _dev(self, t, dtype):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype
                and t.is_contiguous() and t.numel() == self.n):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor of {self.n} entries")
        return ctypes.c_void_p(t.data_ptr())

    def solve(self, f, tol=0.0, out=None, raise_on_error=True, x0=None):
        """u with K u = f; f: CUDA float64 tensor.  x0: optional starting guess
        u_-1 (Algorithm 2 with a nonzero u_-1).  Returns (u, info dict)."""
        u = out if out is not None else torch.empty_like(f)
        res = L.Result()
        if x0 is not None:
            if x0.data_ptr() != u.data_ptr():
                u.copy_(x0)
            s = self._lib.xdcg_solve_x0(self.ctx, self._dev(f, torch.float64),
                                        self._dev(u, torch.float64), float(tol), ctypes.byref(res))
        else:
            s = self._lib.xdcg_solve(self.ctx, self._dev(f, torch.float64),
                                     self._dev(u, torch.float64), float(tol), ctypes.byref(res))
        info = res.as_dict()
        info["status"] = L.STATUS.get(s, s)
        if raise_on_error:
            L.check(s, "xdcg_solve", res.bad_index)
        return u, info

    def solve_batch(self, F, tol=0.0, out=None, raise_on_error=True):
        """U with K U_j = F_j for the rows F_j of F ((m, n) contiguous CUDA float64);
        mixed contexts with max_batch >= m run them as one batched FP32 iteration.
        Returns (U, list of per-column info dicts)."""
        if not (F.is_cuda and F.dtype == torch.float64 and F.is_contiguous() and F.dim() == 2
                and F.shape[1] == self.n):
            raise ValueError(f"expected a contiguous (m, {self.n}) CUDA float64 tensor")
        m = F.shape[0]
        U = out if out is not None else torch.empty_like(F)
        res = (L.Result * m)()
        s = self._lib.xdcg_solve_batch(self.ctx, ctypes.c_void_p(F.data_ptr()),
                                       ctypes.c_void_p(U.data_ptr()), m, float(tol),
                                       ctypes.cast(res, ctypes.c_void_p))
        infos = [r.as_dict() for r in res]
        for i in infos:
            i["status"] = L.STATUS.get(s, s)
        if raise_on_error:
            L.check(s, "xdcg_solve_batch")
        return U, infos

    def history(self):
        """||r_i|| / ||f||, i = 0 .. iterations, of the last FP64 solve."""
        count = ctypes.c_int32(0)
        L.check(self._lib.xdcg_get_history(self.ctx, None, 0, ctypes.byref(count)),
                "xdcg_get_history")
        out = np.empty(count.value)
        if count.value:
            L.check(self._lib.xdcg_get_history(self.ctx, ctypes.c_void_p(out.ctypes.data),
                                               count.value, ctypes.byref(count)),
                    "xdcg_get_history")
        return out

    def solve_host(self, f_host, u_host, tol=0.0):
        """Host-memory solve (copies inside the call); f_host, u_host: float64 arrays
        or pinned CPU tensors of n entries."""
        def ptr(a):
            if isinstance(a, torch.Tensor):
                assert a.dtype == torch.float64 and not a.is_cuda and a.numel() == self.n
                return ctypes.c_void_p(a.data_ptr())
            assert a.dtype == np.float64 and a.size == self.n and a.flags.c_contiguous
            return ctypes.c_void_p(a.ctypes.data)
        res = L.Result()
        L.check(self._lib.xdcg_solve_host(self.ctx, ptr(f_host), ptr(u_host), float(tol),
                                          ctypes.byref(res)), "xdcg_solve_host", res.bad_index)
        return res.as_dict()

    def spmv(self, x, precision="fp64"):
        """y = K x; returns (y, x^T y)."""
        dt = torch.float64 if precision == "fp64" else torch.float32
        y = torch.empty_like(x)
        xty = ctypes.c_double()
        L.check(self._lib.xdcg_spmv(self.ctx, L.XDCG_FP64 if precision == "fp64" else L.XDCG_MIXED,
                                    self._dev(x, dt), self._dev(y, dt), ctypes.byref(xty)),
                "xdcg_spmv")
        return y, xty.value

    def element_sensitivity(self, elements, u, lam, out=None):
        """dJ/dE_e = -lam_e^T Khat_e u_e per element (K lam = dJ/du); u, lam:
        CUDA float64 tensors of n entries; elements: an Elements on the same
        device.  Returns a float64 tensor of one entry per element."""
        out = out if out is not None else torch.empty(elements.n_el, dtype=torch.float64,
                                                      device=u.device)
        if out.numel() != elements.n_el or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out: a contiguous float64 tensor of one entry per element")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())
        L.check(self._lib.xdcg_element_sensitivity(
            self.ctx, elements.n_el, ptr(elements.dof_ptr), ptr(elements.dofs),
            ptr(elements.mat_off), ptr(elements.mats), elements.mats.numel(),
            self._dev(u, torch.float64), self._dev(lam, torch.float64), ptr(out)),
            "xdcg_element_sensitivity")
        return out

    def stiffness_gradient(self, pattern, lam, u, out=None):
        """dJ/dK = -lam u^T at K's stored entries (K lam = dJ/du), in K's
        value layout: one float64 entry per stored value."""
        out = out if out is not None else torch.empty(pattern.nval, dtype=torch.float64,
                                                      device=u.device)
        if out.numel() != pattern.nval or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out: a contiguous float64 tensor of one entry per stored value")
        ptr = lambda t: t.data_ptr()
        m = L.Matrix(pattern.n_nodes, ptr(pattern.dof_ptr), ptr(pattern.row_ptr),
                     ptr(pattern.col), ptr(pattern.val_ptr), None, L.XDCG_DEVICE)
        L.check(self._lib.xdcg_stiffness_gradient(
            self.ctx, ctypes.byref(m), self._dev(lam, torch.float64), self._dev(u, torch.float64),
            ctypes.c_void_p(out.data_ptr())), "xdcg_stiffness_gradient")
        return out

    def precond(self, r):
        """z = A-DEF2 preconditioner applied to r (FP64)."""
        z = torch.empty_like(r)
        L.check(self._lib.xdcg_precond(self.ctx, self._dev(r, torch.float64),
                                       self._dev(z, torch.float64)), "xdcg_precond")
        return z

    def coarse_matrix(self):
        E = np.empty((self.k, self.k))
        L.check(self._lib.xdcg_coarse_matrix(self.ctx, ctypes.c_void_p(E.ctypes.data)),
                "xdcg_coarse_matrix")
        return E

    def close(self):
        if self.ctx:
            self._lib.xdcg_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
