"""Several systems, each with several load cases, solved together: the
systems of successive crack-front positions in a propagation sweep.

Every system has its own context (its K, Z, block factors and coarse
operator differ with the crack front), and its load cases run as one batched
FP32 iteration.  By default each system's batched solve is issued from a host
thread of its own on its own stream, so the systems' kernels overlap on the
GPU (the library releases the GIL through ctypes and blocks only on its own
stream).  fused=True runs them as one xdcg_solve_systems call instead: every
iteration is one launch per kernel over all systems' blocks, and a system
whose columns wait for their residual replacement is held while the
replacement runs on its own stream.  Every mode gives the same bits per
column (fixed partitions and reduction orders in every kernel, and columns
that advance independently).
"""
import concurrent.futures as cf

import torch

from .solver import Solver


def make_solvers(problems, max_batch=8, precision="mixed", **kw):
    """One context per problem (mixed precision by default), each on a
    stream of its own."""
    return [Solver.from_problem(P, precision=precision, max_batch=max_batch,
                                stream=torch.cuda.Stream(), **kw) for P in problems]


def solve_systems(solvers, loads, tol, outs=None, concurrent=True, raise_on_error=True,
                  fused=False):
    """solvers[i].solve_batch(loads[i], tol) for every system i.

    loads[i]: (m_i, n_i) contiguous CUDA float64 tensor of system i's load
    cases; outs: optional matching output tensors.  Inputs must be ready on
    the device (the call synchronises the device first).  fused=True (two or
    more mixed batched contexts): one xdcg_solve_systems call; otherwise
    concurrent=True runs each system's solve_batch from a thread of its own
    and concurrent=False one after another.  Returns [(U_i, infos_i)]."""
    if len(solvers) != len(loads):
        raise ValueError("one load tensor per solver")
    outs = outs if outs is not None else [torch.empty_like(F) for F in loads]
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if fused and len(solvers) > 1:
        return _solve_fused(solvers, loads, tol, outs, raise_on_error)

    def run(i):
        return solvers[i].solve_batch(loads[i], tol=tol, out=outs[i],
                                      raise_on_error=raise_on_error)

    if not concurrent or len(solvers) == 1:
        return [run(i) for i in range(len(solvers))]
    with cf.ThreadPoolExecutor(len(solvers)) as ex:
        return list(ex.map(run, range(len(solvers))))


def _solve_fused(solvers, loads, tol, outs, raise_on_error):
    import ctypes

    from . import _lib as L
    ns = len(solvers)
    for S, F, U in zip(solvers, loads, outs):
        if not (F.is_cuda and F.dtype == torch.float64 and F.is_contiguous() and F.dim() == 2
                and F.shape[1] == S.n and U.shape == F.shape and U.is_contiguous()):
            raise ValueError(f"expected contiguous (m, {S.n}) CUDA float64 tensors")
    ctxs = (ctypes.c_void_p * ns)(*[S.ctx.value for S in solvers])
    fp = (ctypes.c_void_p * ns)(*[F.data_ptr() for F in loads])
    up = (ctypes.c_void_p * ns)(*[U.data_ptr() for U in outs])
    ms = (ctypes.c_int32 * ns)(*[F.shape[0] for F in loads])
    res = (L.Result * sum(F.shape[0] for F in loads))()
    st = (ctypes.c_int32 * ns)()
    lib = solvers[0]._lib
    s = lib.xdcg_solve_systems(ctypes.cast(ctxs, ctypes.c_void_p), ns,
                               ctypes.cast(fp, ctypes.c_void_p), ctypes.cast(up, ctypes.c_void_p),
                               ctypes.cast(ms, ctypes.c_void_p), float(tol),
                               ctypes.cast(res, ctypes.c_void_p), ctypes.cast(st, ctypes.c_void_p))
    if raise_on_error:
        L.check(s, "xdcg_solve_systems")
    out, k = [], 0
    for i, F in enumerate(loads):
        infos = [res[k + j].as_dict() for j in range(F.shape[0])]
        for d in infos:
            d["status"] = L.STATUS.get(st[i] if s == 0 else s, s)
        k += F.shape[0]
        out.append((outs[i], infos))
    return out


def transfer_index(dof_prev, kind_prev, dof_next, kind_next):
    """Dof maps (src, dst) that carry a solution of one crack front's system
    into the numbering of the next front's system on the same nodes: each
    node's standard dofs, and its enriched dofs where the node keeps its
    enrichment; every other dof of the next system starts at 0."""
    import numpy as np
    dp, dn = np.asarray(dof_prev, np.int64), np.asarray(dof_next, np.int64)
    kp, kn = np.asarray(kind_prev), np.asarray(kind_next)
    if dp.size != dn.size:
        raise ValueError("the two systems must share their nodes")
    bp, bn = np.diff(dp), np.diff(dn)
    width = np.where(kp == kn, np.minimum(bp, bn), 3)
    src = np.concatenate([dp[:-1][width >= w] + w - 1 for w in range(1, 16)] or [[]])
    dst = np.concatenate([dn[:-1][width >= w] + w - 1 for w in range(1, 16)] or [[]])
    return src.astype(np.int64), dst.astype(np.int64)


def transfer_guess(u_prev, maps, n_next):
    """The previous front's solution in the next system's numbering (a warm
    start, u_-1 of Algorithm 2, for xdcg_solve_x0)."""
    src, dst = maps
    out = torch.zeros(n_next, dtype=u_prev.dtype, device=u_prev.device)
    out[torch.as_tensor(dst, device=u_prev.device)] = u_prev[torch.as_tensor(src,
                                                                             device=u_prev.device)]
    return out
