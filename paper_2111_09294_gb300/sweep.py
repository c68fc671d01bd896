"""Several systems, each with several load cases, solved together: the
systems of successive crack-front positions in a propagation sweep.

Every system has its own context on its own CUDA stream (its K, Z, block
factors and coarse operator differ with the crack front), and its load cases
run as one batched solve on that context.  The systems' calls are issued
from one host thread each (the library releases the GIL through ctypes and
blocks only on its own stream), so their kernels overlap on the GPU: the
small per-system kernels of the FP32 iteration leave most of the GPU idle
when a system runs alone.  Results are bit-for-bit those of the same solves
run one after another (fixed partitions and reduction orders in every
kernel).
"""
import concurrent.futures as cf

import torch

from .solver import Solver


def make_solvers(problems, max_batch=8, precision="mixed", **kw):
    """One context per problem (mixed precision by default), each on a
    stream of its own."""
    return [Solver.from_problem(P, precision=precision, max_batch=max_batch,
                                stream=torch.cuda.Stream(), **kw) for P in problems]


def solve_systems(solvers, loads, tol, outs=None, concurrent=True, raise_on_error=True):
    """solvers[i].solve_batch(loads[i], tol) for every system i.

    loads[i]: (m_i, n_i) contiguous CUDA float64 tensor of system i's load
    cases; outs: optional matching output tensors.  Inputs must be ready on
    the device (the call synchronises the device first).  concurrent=False
    runs the systems one after another.  Returns [(U_i, infos_i)]."""
    if len(solvers) != len(loads):
        raise ValueError("one load tensor per solver")
    outs = outs if outs is not None else [torch.empty_like(F) for F in loads]
    if torch.cuda.is_available():
        torch.cuda.synchronize()

    def run(i):
        return solvers[i].solve_batch(loads[i], tol=tol, out=outs[i],
                                      raise_on_error=raise_on_error)

    if not concurrent or len(solvers) == 1:
        return [run(i) for i in range(len(solvers))]
    with cf.ThreadPoolExecutor(len(solvers)) as ex:
        return list(ex.map(run, range(len(solvers))))
