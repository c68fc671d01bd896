"""Host-side logic without a GPU: the multi-process replica path of bench.py
(two gloo ranks on 127.0.0.1) and the concurrent issue of several systems'
solves (paper_2111_09294_gb300.sweep) with stand-in solvers."""
import os
import socket
import threading
import time

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import types

    import bench
    w, r, local, pg = bench.dist_setup(types.SimpleNamespace(impl="reference"))
    bench.barrier(pg)
    # each rank's time differs; the job's is the slowest rank's
    slowest = bench.max_over_ranks(pg, 10.0 + r)
    bench.barrier(pg)
    q.put((r, w, local, slowest))
    pg.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank_over_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(o[0] for o in out) == [0, 1]
    assert all(o[1] == 2 and o[2] == o[0] and o[3] == 11.0 for o in out)


class _FakeSolver:
    """Stands in for a Solver: solve_batch doubles its input after a delay
    and records the threads that ran it."""

    def __init__(self, delay, fail=False):
        self.delay, self.fail, self.threads = delay, fail, []

    def solve_batch(self, F, tol=0.0, out=None, raise_on_error=True):
        self.threads.append(threading.get_ident())
        time.sleep(self.delay)
        if self.fail:
            raise RuntimeError("solve failed")
        out.copy_(2 * F)
        return out, [{"iterations": 1, "tol": tol}] * F.shape[0]


def test_sweep_keeps_system_order_and_overlaps_calls():
    from paper_2111_09294_gb300 import sweep as S
    solvers = [_FakeSolver(0.6), _FakeSolver(0.15), _FakeSolver(0.3)]
    loads = [torch.full((2, 3), float(i)) for i in range(3)]
    t0 = time.perf_counter()
    res = S.solve_systems(solvers, loads, 1e-8)
    concurrent = time.perf_counter() - t0
    for i, (U, infos) in enumerate(res):
        assert torch.equal(U, 2 * loads[i]) and len(infos) == 2 and infos[0]["tol"] == 1e-8
    # one host thread per system: the calls overlap
    assert len({s.threads[0] for s in solvers}) == 3
    assert concurrent < 0.9           # one after another takes 1.05 s
    seq = S.solve_systems(solvers, loads, 1e-8, concurrent=False)
    assert all(torch.equal(a[0], b[0]) for a, b in zip(res, seq))
    assert len({s.threads[1] for s in solvers}) == 1


def test_sweep_reports_a_failed_system():
    from paper_2111_09294_gb300 import sweep as S
    solvers = [_FakeSolver(0.0), _FakeSolver(0.0, fail=True)]
    with pytest.raises(RuntimeError, match="solve failed"):
        S.solve_systems(solvers, [torch.zeros(1, 2), torch.zeros(1, 2)], 1e-8)
    with pytest.raises(ValueError):
        S.solve_systems(solvers, [torch.zeros(1, 2)], 1e-8)
    # the fused call takes contiguous (m, n) CUDA float64 loads only
    solvers[0].n = solvers[1].n = 2
    with pytest.raises(ValueError):
        S.solve_systems(solvers, [torch.zeros(1, 2), torch.zeros(1, 2)], 1e-8, fused=True)


def test_profiled_traffic_is_reported_only_for_the_captured_kernel(tmp_path):
    # the bench line's roofline traffic comes from a committed ncu summary,
    # and only while the kernel's sources hash to the recorded value and the
    # timed product runs the captured pipeline shape
    import bench
    sha = bench.kernel_source_sha(bench.SPMV_SOURCES)
    p = tmp_path / "summary.md"
    p.write_text(f"traffic_bytes_per_launch: 181941248\nkernel_source_sha256: {sha}\n"
                 "kernel_shape: 5\n")
    assert bench.profiled_traffic(bench.SPMV_SOURCES, str(p), 5) == 181941248.0
    assert bench.profiled_traffic(bench.SPMV_SOURCES, str(p), 0) is None
    p.write_text("traffic_bytes_per_launch: 181941248\nkernel_source_sha256: 000000000000\n"
                 "kernel_shape: 5\n")
    assert bench.profiled_traffic(bench.SPMV_SOURCES, str(p), 5) is None
    p.write_text(f"traffic_bytes_per_launch: 181941248\nkernel_source_sha256: {sha}\n")
    assert bench.profiled_traffic(bench.SPMV_SOURCES, str(p), 5) is None
    assert bench.spmv_kernel_name(5).startswith("k_spmv_lean<false, 5>")
    assert bench.spmv_kernel_name(0).startswith("k_spmv<float, false, 0>")
