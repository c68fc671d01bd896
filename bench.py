"""Benchmark: time to ||f - K u|| / ||f|| <= 1e-8 on the 48^3 two-crack cube.

Default arm: the GPU library.  One step = one full solve (all steps of the
hot path: Algorithm 2 start, A-DEF2 PCG iterations, FP64 residual replacement
for the mixed path) with the load vector already resident in HBM; L2 is flushed
(a 256 MiB write) before every timed step, outside the step's events.
Reported: mixed (FP32 PCG / FP64 residual replacement) solve time as the value, the
plain FP64 solve time and the mixed solve with an FP64 coarse solve beside it,
iterations (the oracle's too), SpMV bandwidth against the measured HBM copy
bandwidth, the FP64 SpMV against the measured FP64 rate, one full FP64 CPU
oracle solve on 1 thread and on all host cores, an end-to-end figure through
the host-memory entry point, and the batched, differentiable and
propagation-sweep workloads.

--impl reference: the CPU oracle as the reference arm (same metric and
workload, each step a bounded sample of oracle iterations scaled to the
oracle's own iteration count).
"""
import argparse
import json
import os
import re
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import hashlib

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to ‖r‖/‖f‖≤1e-8: mixed vs FP64 DPCG on GB300; SpMV GB/s vs HBM peak"
WORKLOAD = "cube48_two_cracks"
TOL = 1e-8
FALLBACK_HBM = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def kernel_source_sha(files):
    """First 12 hex digits of the SHA-256 of the kernel's source files, in order."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2111_09294_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


SPMV_SOURCES = ("spmv.cu", "spmv_cfg.cuh", "tma.cuh", "pdl.cuh", "cache.cuh")


def profiled_traffic(kernel_files, summary, shape):
    """Per-launch DRAM bytes of the FP32 SpMV from the committed ncu summary,
    or None when the kernel's sources changed since the capture or the
    capture is of another pipeline shape than the one timed."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]{12})", txt)
    k = re.search(r"kernel_shape:\s*([0-9]+)", txt)
    if not m or not h or not k:
        return None
    if kernel_source_sha(kernel_files) != h.group(1) or int(k.group(1)) != shape:
        return None
    return float(m.group(1))


def spmv_kernel_name(shape):
    """The FP32 SpMV kernel a pipeline shape runs (shapes 5-7: the lean kernel)."""
    return (f"k_spmv_lean<false, {shape}>" if shape >= 5 else
            f"k_spmv<float, false, {shape}>") + " (inner FP32 SpMV)"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v, device=None):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_full_solve(workload):
    """One full FP64 oracle solve to 1e-8 (set-up timed separately); runs in
    the process whose BLAS thread count the caller fixed."""
    import xfem_inputs as X
    from oracle import adef2 as O
    P = X.make(workload)
    t0 = time.perf_counter()
    K, M, C = O.setup(P)
    t1 = time.perf_counter()
    r = O.adef2_pcg(K, P.f, M, C, tol=TOL)
    t2 = time.perf_counter()
    return {"ms": (t2 - t1) * 1e3, "setup_ms": (t1 - t0) * 1e3, "iterations": r.iterations,
            "rel_res_true": float(np.linalg.norm(P.f - K @ r.u) / np.linalg.norm(P.f))}


def oracle_timing(workload, threads):
    """oracle_full_solve in a fresh Python process with `threads` BLAS/OpenMP
    threads (the thread count is fixed when numpy loads, so each count needs a
    process of its own; no CUDA is touched there)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-solve",
                        "--workload", workload], env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"oracle run failed: {r.stderr[-300:]}")
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["threads"] = threads
    return out


def fp64_peak_tflops(dev):
    """Measured FP64 rate of this GPU: a cuBLAS DGEMM (4096^3, 2 n^3 flops),
    best of 5 after a warm-up, CUDA events."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import xfem_inputs as X
    from oracle import adef2 as O
    P = X.make(args.workload)
    K, M, C = O.setup(P)
    full = O.adef2_pcg(K, P.f, M, C, tol=TOL)
    its = full.iterations
    times, steps_ms = [], []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = O.adef2_pcg(K, P.f, M, C, tol=TOL, maxit=args.sample_iters)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt / r.iterations * its * 1e3)
            steps_ms.append(dt * 1e3)
    # value: one full solve, estimated from the step's sample; ms_per_step: the
    # sample a step actually ran (what the timed region took)
    value = float(np.mean(times))
    sample = (f"{args.sample_iters} oracle iterations per step ({float(np.mean(steps_ms)):.0f} ms "
              f"each), scaled to the oracle's {its} iterations to 1e-8 (setup excluded)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": float(np.mean(steps_ms)), "value_per": "one full solve (estimated)",
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_dict(P, C.k, args.workload),
           "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "oracle_iterations": its}
    print(json.dumps(out))


DESCRIPTIONS = {
    "cube8_edge": "8^3 hexes, planar edge crack, r_e=0.15, 2^3 boxes",
    "cube24_ellipse": "24^3 hexes, tilted warped elliptical crack, r_e=0.08, 4^3 boxes",
    "cube48_two_cracks": "48^3 hexes, penny r=0.2 + edge crack depth 0.25, warped, r_e=0.05, "
                         "8^3 boxes",
    "cube64_penny_lognormal": "64^3 hexes, warped penny r=0.3, r_e=0.05, 8^3 boxes, element "
                              "moduli log-normal(0, 0.3)",
}


def config_dict(P, k, workload):
    return {"workload": f"{workload}: {DESCRIPTIONS.get(workload, '')}",
            "n_dofs": int(P.n), "n_nodes": int(P.n_nodes), "enriched_dofs":
            int(P.n_heaviside_dofs + P.n_tip_dofs), "coarse_k": int(k), "tol": TOL,
            "l2": "flushed (256 MiB write) before every timed step"}


def optional(fn):
    """An extra measurement that fails is reported in the line, not fatal to it."""
    try:
        return fn()
    except Exception as e:   # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def run_ours(args):
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import xfem_inputs as X
    from paper_2111_09294_gb300 import Solver
    P = X.make(args.workload)
    stream = torch.cuda.current_stream(dev)
    # the solves timed for the value carry no events inside (events between
    # kernels would break their programmatic dependent launches); separate
    # solvers with CUDA events around every SpMV give the SpMV's own time
    # every SpMV pipeline shape timed at set-up on this matrix, the fastest kept
    at = bool(args.autotune)
    mixed = Solver.from_problem(P, precision="mixed", inner_tol=args.inner_tol, autotune=at)
    fp64 = Solver.from_problem(P, precision="fp64", autotune=at)
    mixed_c64 = Solver.from_problem(P, precision="mixed", inner_tol=args.inner_tol,
                                    coarse_fp64=True, autotune=at)
    mixed_t = Solver.from_problem(P, precision="mixed", time_spmv=True, inner_tol=args.inner_tol,
                                  autotune=at)
    fp64_t = Solver.from_problem(P, precision="fp64", time_spmv=True, autotune=at)
    # the same solves with their iterations replayed as recorded CUDA graphs
    mixed_g = Solver.from_problem(P, precision="mixed", inner_tol=args.inner_tol, autotune=at,
                                  graph=True)
    fp64_g = Solver.from_problem(P, precision="fp64", autotune=at, graph=True)
    f = torch.tensor(P.f, device=dev)
    u = torch.empty_like(f)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(solver, steps, warmup, collect):
        for _ in range(warmup):
            solver.solve(f, tol=TOL, out=u)
        ms, infos = [], []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = solver.solve(f, tol=TOL, out=u)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        return ms, infos

    torch.cuda.synchronize()
    barrier(pg)
    clocks = ClockSampler(local)
    clocks.start()
    ms_mixed, inf_mixed = timed(mixed, args.steps, args.warmup, True)
    torch.cuda.synchronize()
    barrier(pg)
    ms_fp64, inf_fp64 = timed(fp64, args.steps, args.warmup, True)
    torch.cuda.synchronize()
    barrier(pg)
    ms_c64, inf_c64 = timed(mixed_c64, args.steps, args.warmup, True)
    torch.cuda.synchronize()
    barrier(pg)
    ms_mg, inf_mg = timed(mixed_g, args.steps, args.warmup, True)
    ms_fg, inf_fg = timed(fp64_g, args.steps, args.warmup, True)
    torch.cuda.synchronize()
    barrier(pg)
    # SpMV kernel time: a timed pass of the same solves with events around each SpMV
    _, inf_mixed_t = timed(mixed_t, args.steps, 1, True)
    _, inf_fp64_t = timed(fp64_t, args.steps, 1, True)
    torch.cuda.synchronize()
    barrier(pg)
    # clocks sampled over all timed passes (the value's alone is tens of ms)
    clk = clocks.stop()
    t_mixed = max_over_ranks(pg, float(np.mean(ms_mixed)), dev)
    t_fp64 = max_over_ranks(pg, float(np.mean(ms_fp64)), dev)
    res_true = max(i["rel_res_true"] for i in inf_mixed)
    assert res_true <= TOL, res_true

    # end to end through the host-memory entry point (pinned buffers)
    fh = torch.tensor(P.f, dtype=torch.float64).pin_memory()
    uh = torch.empty(P.n, dtype=torch.float64).pin_memory()
    for _ in range(max(1, args.warmup)):
        mixed.solve_host(fh, uh, tol=TOL)
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mixed.solve_host(fh, uh, tol=TOL)
        e2e.append((time.perf_counter() - t0) * 1e3)
    t_e2e = max_over_ranks(pg, float(np.mean(e2e)), dev)

    if rank != 0:
        return
    # per-kernel time per iteration, from separate solves with CUDA events
    # around every kernel of the loop (outside the timed region)
    phases = {}
    for prec, names in (("mixed", ("spmv", "restrict_update", "coarse", "prolong")),
                        ("fp64", ("spmv", "update", "restrict", "coarse", "prolong"))):
        diag = Solver.from_problem(P, precision=prec, time_spmv="kernels",
                                   inner_tol=args.inner_tol)
        diag.solve(f, tol=TOL, out=u)
        flush.zero_()
        _, dinf = diag.solve(f, tol=TOL, out=u)
        nt = max(dinf["n_phase_timed"], 1)
        phases[prec] = {nm: round(1e3 * t / nt, 2) for nm, t in zip(names, dinf["t_phase_ms"])}
        if prec == "mixed":
            di = diag.info
            nbytes = {"spmv": di["spmv_bytes_fp32"], "restrict_update": di["restrict_bytes_fp32"],
                      "coarse": di["coarse_bytes_fp32"], "prolong": di["prolong_bytes_fp32"]}
            # the fused iteration has no separate prolongation (0 us, 0 bytes)
            phases["mixed_gbs"] = {nm: round(nbytes[nm] / (phases[prec][nm] * 1e-6) / 1e9)
                                   for nm in names if phases[prec][nm] > 0 and nbytes[nm] > 0}
        diag.close()
    # several load cases of the same crack configuration: one batched FP32 run
    # against the same columns solved one after another (outside the value)
    def measure_batch():
        m = args.batch
        Fb = torch.tensor(X.load_cases(P, m, seed=0), device=dev)
        Ub = torch.empty_like(Fb)
        bsol = Solver.from_problem(P, precision="mixed", inner_tol=args.inner_tol, max_batch=m)
        for _ in range(max(1, args.warmup)):
            bsol.solve_batch(Fb, tol=TOL, out=Ub)
        tb, t1, binfs = [], [], None
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, binfs = bsol.solve_batch(Fb, tol=TOL, out=Ub)
            e1.record(stream)
            e1.synchronize()
            tb.append(e0.elapsed_time(e1))
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for j in range(m):
                mixed.solve(Fb[j], tol=TOL, out=u)
            e1.record(stream)
            e1.synchronize()
            t1.append(e0.elapsed_time(e1))
        rmax = max(i["rel_res_true"] for i in binfs)
        assert rmax <= TOL, rmax
        tb_ms, t1_ms = float(np.mean(tb)), float(np.mean(t1))
        batch = {"rhs": m, "ms": tb_ms, "rhs_per_s": m / tb_ms * 1e3,
                 "ms_one_by_one": t1_ms, "speedup_vs_one_by_one": t1_ms / tb_ms,
                 "iterations_max": max(i["iterations"] for i in binfs),
                 "rel_res_true_max": rmax,
                 "loads": "seeded tractions on z = 1: shear and tension, |t_i| ~ U[0.5, 1.5]"}
        bsol.close()
        return batch
    # differentiable solve: forward u = K^-1 f and the adjoint backward for
    # the compliance J = f.u (dJ/df and dJ/dE_e for every element's modulus),
    # mixed against FP64 (outside the value)
    def measure_fwd_bwd():
        from paper_2111_09294_gb300 import Elements
        from paper_2111_09294_gb300.autograd import solve as dsolve
        elems = Elements.from_dict(X.element_data(P), dev)
        young = torch.tensor(P.young, device=dev)
        fwd_bwd = {}
        for name, solver in (("mixed", mixed), ("fp64", fp64)):
            ts = []
            for it in range(args.warmup + args.steps):
                fg = f.clone().requires_grad_(True)
                yg = young.clone().requires_grad_(True)
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                J = (fg * dsolve(solver, fg, TOL, young=yg, elements=elems)).sum()
                J.backward()
                e1.record(stream)
                e1.synchronize()
                if it >= args.warmup:
                    ts.append(e0.elapsed_time(e1))
            # median and mean of the timed steps (the median is robust to a
            # one-off host stall inside autograd)
            fwd_bwd[name + "_ms"] = float(np.median(ts))
            fwd_bwd[name + "_ms_mean"] = float(np.mean(ts))
        # the element kernel alone (all elements, one launch)
        lam_t = torch.randn(P.n, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            mixed.element_sensitivity(elems, u, lam_t)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            mixed.element_sensitivity(elems, u, lam_t)
        e1.record(stream)
        e1.synchronize()
        # per call, including the call's status read (a stream synchronisation)
        fwd_bwd["element_call_ms"] = e0.elapsed_time(e1) / max(args.steps, 1)
        fwd_bwd["elements"] = elems.n_el
        if args.chain_steps > 1 and args.workload == X.STEPS64[0]:
            fwd_bwd["propagation_steps"] = optional(lambda: chain(args.chain_steps))
        fwd_bwd["speedup_mixed_vs_fp64"] = fwd_bwd["fp64_ms"] / fwd_bwd["mixed_ms"]
        fwd_bwd["loss"] = ("compliance J = f . u; backward = adjoint solve to the same tol, then "
                           "dJ/df and dJ/dE_e for every element")
        return fwd_bwd
    # total compliance over successive crack-front positions of the 64^3
    # log-normal workload, u recomputed in the backward instead of stored
    def chain(nsteps):
        from paper_2111_09294_gb300 import Elements
        from paper_2111_09294_gb300.autograd import compliance_steps
        Ps = X.make_many(X.STEPS64[:nsteps])
        elems = [Elements.from_dict(X.element_data(Pi), dev) for Pi in Ps]
        young = torch.tensor(Ps[0].young, device=dev)
        out = {"steps": nsteps, "n_dofs": [int(Pi.n) for Pi in Ps],
               "loss": "sum over steps of f_s . u_s; u_s recomputed in the backward"}
        for name in ("mixed", "fp64"):
            sols = [Solver.from_problem(Pi, precision=name, inner_tol=args.inner_tol)
                    for Pi in Ps]
            loads = [torch.tensor(Pi.f, device=dev) for Pi in Ps]
            ts = []
            for it in range(max(1, args.warmup) + args.steps):
                fs = [l.clone().requires_grad_(True) for l in loads]
                yg = young.clone().requires_grad_(True)
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                J = compliance_steps(sols, fs, TOL, young=yg, elements=elems)
                J.backward()
                e1.record(stream)
                e1.synchronize()
                if it >= max(1, args.warmup):
                    ts.append(e0.elapsed_time(e1))
            out[name + "_ms"] = float(np.median(ts))
            for sl in sols:
                sl.close()
        out["speedup_mixed_vs_fp64"] = out["fp64_ms"] / out["mixed_ms"]
        return out

    # a propagation sweep: --sweep systems of the 32^3 inclined-penny sweep,
    # 8 load cases each, every system a batched mixed solve: concurrent (a
    # host thread and a stream per system, the default), fused (one launch
    # per kernel over all systems) and one after another (outside the value)
    def measure_sweep():
        from paper_2111_09294_gb300 import sweep as S
        Ps = X.make_many(X.SWEEP[:args.sweep])
        ssol = S.make_solvers(Ps, max_batch=8)
        gsol = S.make_solvers(Ps, max_batch=8, graph=True)
        Fs = [torch.tensor(X.load_cases(Pi, 8, seed=100 + i), device=dev)
              for i, Pi in enumerate(Ps)]
        Us = [torch.empty_like(Fi) for Fi in Fs]
        modes = {"concurrent": (ssol, {}), "fused": (ssol, {"fused": True}),
                 "one_after_another": (ssol, {"concurrent": False}),
                 "concurrent_graph": (gsol, {}), "fused_graph": (gsol, {"fused": True})}
        times, res = {}, {}
        for name, (sol_, kw) in modes.items():
            for _ in range(max(1, args.warmup)):
                S.solve_systems(sol_, Fs, TOL, outs=Us, **kw)
            ts_ = []
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                out_ = S.solve_systems(sol_, Fs, TOL, outs=Us, **kw)
                ts_.append((time.perf_counter() - t0) * 1e3)
            # the outputs are shared by the modes: keep this mode's
            res[name] = [(U_.clone(), inf_) for U_, inf_ in out_]
            times[name] = float(np.mean(ts_))
        infos = [i for _, inf in res["concurrent"] for i in inf]
        assert max(i["rel_res_true"] for i in infos) <= TOL
        same = all(torch.equal(a[0], b[0]) for a, b in zip(res["fused"], res["concurrent"]))
        same_g = all(torch.equal(a[0], b[0]) and torch.equal(a[0], c[0]) for a, b, c in
                     zip(res["fused_graph"], res["concurrent_graph"], res["concurrent"]))
        sweep = {"systems": len(Ps), "rhs_per_system": 8,
                 "n_dofs": [int(Pi.n) for Pi in Ps], "ms": times["concurrent"],
                 "ms_fused": times["fused"],
                 "ms_one_after_another": times["one_after_another"],
                 "speedup_vs_one_after_another": times["one_after_another"] / times["concurrent"],
                 "fused_same_bits": same,
                 "ms_concurrent_graph": times["concurrent_graph"],
                 "ms_fused_graph": times["fused_graph"], "graph_same_bits": same_g,
                 "systems_rhs_per_s": len(Ps) * 8 / times["concurrent"] * 1e3,
                 "iterations_max": max(i["iterations"] for i in infos),
                 "iterations_mean": float(np.mean([i["iterations"] for i in infos])),
                 "rel_res_true_max": max(i["rel_res_true"] for i in infos),
                 "timing": "host wall clock around the calls (each returns after its work)"}
        for s_ in ssol + gsol:
            s_.close()
        return sweep

    # the paper's own block choice, one block-Jacobi block per subdomain
    # (enriched dofs included), on the same system numbered box by box:
    # FP64 and mixed solves against node blocks in that numbering (outside
    # the value)
    def measure_subdomain_blocks():
        P2, bp = X.by_subdomain(P)
        f2 = torch.tensor(P2.f, device=dev)
        u2 = torch.empty_like(f2)
        out = {"blocks": len(bp) - 1, "block_dofs_max": int(np.max(np.diff(bp))),
               "block_dofs_mean": float(np.mean(np.diff(bp)))}
        for prec in ("mixed", "fp64"):
            for kind, kw in (("subdomain", {"blocks": bp}), ("node", {})):
                sol = Solver.from_problem(P2, precision=prec, inner_tol=args.inner_tol, **kw)
                for _ in range(max(1, args.warmup)):
                    sol.solve(f2, tol=TOL, out=u2)
                ts, inf = [], None
                for _ in range(args.steps):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    _, inf = sol.solve(f2, tol=TOL, out=u2)
                    e1.record(stream)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                assert inf["rel_res_true"] <= TOL * 1.05, inf
                out[f"{prec}_{kind}"] = {"ms": float(np.mean(ts)), "iterations": inf["iterations"],
                                         "setup_ms": sol.info["t_setup_ms"],
                                         "iter_bytes": sol.info["iter_bytes_fp32" if prec == "mixed"
                                                                else "iter_bytes_fp64"]}
                if kind == "subdomain":
                    out["block_entries"] = sol.info["block_entries"]
                sol.close()
        return out

    blocks_row = optional(measure_subdomain_blocks) if args.subdomain_blocks else None

    # iterations against n at a fixed subdomain size (boxes of 6^3 hexes, the
    # 24^3 case's crack at 12^3 .. 48^3 hexes): GPU counts and times
    def measure_trend():
        rows = []
        for name in X.TREND:
            Pt = X.make(name)
            ft = torch.tensor(Pt.f, device=dev)
            row = {"workload": name, "n": int(Pt.n), "n_sub": int(Pt.n_sub),
                   "n_per_sub": int(Pt.n // Pt.n_sub)}
            for prec in ("fp64", "mixed"):
                sol = Solver.from_problem(Pt, precision=prec)
                sol.solve(ft, tol=TOL)
                _, inf = sol.solve(ft, tol=TOL)
                row[f"iterations_{prec}"] = inf["iterations"]
                row[f"ms_{prec}"] = inf["t_solve_ms"]
                sol.close()
            rows.append(row)
        return rows

    trend = optional(measure_trend) if args.trend else None
    # the sweep's crack fronts one after another, as a propagation runs them:
    # each front's set-up fresh and as an update of the previous front's
    # context (unchanged node factors and E^-1 carried over), and its
    # unit-tension solve from zero and warm-started from the previous front's
    # solution (outside the value)
    def measure_sequence():
        from paper_2111_09294_gb300.sweep import transfer_guess, transfer_index
        Ps = X.make_many(X.SWEEP[:args.sweep])
        rows, prev, uprev, Pprev = [], None, None, None
        for Pi in Ps:
            fresh = Solver.from_problem(Pi, precision="mixed", inner_tol=args.inner_tol)
            t_fresh = fresh.info["t_setup_ms"]
            fresh.close()
            sol = Solver.from_problem(Pi, precision="mixed", inner_tol=args.inner_tol, prev=prev)
            fi = torch.tensor(Pi.f, device=dev)
            ucold, icold = sol.solve(fi, tol=TOL)
            row = {"n": int(Pi.n), "setup_fresh_ms": t_fresh, "setup_update_ms":
                   sol.info["t_setup_ms"] if prev is not None else None,
                   "reused_node_factors": sol.info["reused_node_factors"],
                   "iterations_cold": icold["iterations"], "ms_cold": icold["t_solve_ms"]}
            if prev is not None:
                guess = transfer_guess(uprev, transfer_index(Pprev.dof_ptr, Pprev.kind,
                                                             Pi.dof_ptr, Pi.kind), Pi.n)
                _, iw = sol.solve(fi, tol=TOL, x0=guess)
                assert iw["rel_res_true"] <= TOL * 1.05, iw
                row.update(iterations_warm=iw["iterations"], ms_warm=iw["t_solve_ms"])
                prev.close()
            rows.append(row)
            prev, uprev, Pprev = sol, ucold.clone(), Pi
        prev.close()
        upd = [r["setup_update_ms"] for r in rows[1:]]
        return {"fronts": rows, "setup_fresh_ms_total": sum(r["setup_fresh_ms"] for r in rows),
                "setup_update_ms_total": rows[0]["setup_fresh_ms"] + sum(upd),
                "solve_cold_ms_total": sum(r["ms_cold"] for r in rows[1:]),
                "solve_warm_ms_total": sum(r["ms_warm"] for r in rows[1:]),
                "note": "mixed, unit tension, tol 1e-8; totals over fronts 1..15 for the solves"}

    def graph_row():
        # the value's solves with their iterations replayed as CUDA graphs
        # (xdcg_options.graph); the bits match when both contexts run the
        # same SpMV shape (the autotuner may pick another on a close call)
        same = {}
        for name, a, b in (("mixed", mixed, mixed_g), ("fp64", fp64, fp64_g)):
            if a.info["spmv_shape_fp32"] != b.info["spmv_shape_fp32"] or \
                    a.info["spmv_shape_fp64"] != b.info["spmv_shape_fp64"]:
                same[name] = None
                continue
            ua, _ = a.solve(f, tol=TOL)
            ub, _ = b.solve(f, tol=TOL)
            same[name] = bool(torch.equal(ua, ub))
        return {"mixed_ms": max_over_ranks(pg, float(np.mean(ms_mg)), dev),
                "fp64_ms": max_over_ranks(pg, float(np.mean(ms_fg)), dev),
                "mixed_iterations": inf_mg[-1]["iterations"],
                "fp64_iterations": inf_fg[-1]["iterations"],
                "graph_launches_per_solve_mixed": inf_mg[-1]["n_graph_launches"],
                "rel_res_true_mixed": max(i["rel_res_true"] for i in inf_mg),
                "same_bits_as_stream_launches": same,
                "note": "8 iterations per graph launch; timed like the value"}

    def iteration_gbs():
        # effective bandwidth of whole iterations: one iteration's algorithmic
        # bytes times the iterations, over the solve time (which also holds the
        # start and, for the mixed path, the FP64 residual evaluations)
        its_m = inf_mixed[-1]["iterations"]
        gm = info["iter_bytes_fp32"] * its_m / (t_mixed * 1e-3) / 1e9
        gf = fp64.info["iter_bytes_fp64"] * its_fp64 / (t_fp64 * 1e-3) / 1e9
        pk = peaks()[0]
        return {"mixed": gm, "mixed_frac": gm / pk, "fp64": gf, "fp64_frac": gf / pk,
                "iter_bytes_fp32": info["iter_bytes_fp32"],
                "iter_bytes_fp64": fp64.info["iter_bytes_fp64"], "unit": "GB/s"}

    sequence = optional(measure_sequence) if args.sweep > 1 else None
    batch = optional(measure_batch) if args.batch > 0 else None
    fwd_bwd = optional(measure_fwd_bwd)
    sweep = optional(measure_sweep) if args.sweep > 0 else None
    info = mixed.info
    n_sp = sum(i["n_spmv_timed"] for i in inf_mixed_t)
    t_sp = sum(i["t_spmv_ms"] for i in inf_mixed_t)
    spmv_ms = t_sp / max(n_sp, 1)
    # algorithmic bytes on the node-blocked matrix (one index per node block);
    # the kernel's own chunked layout moves spmv_bytes_fp32 (one index per 3x3)
    achieved = info["spmv_alg_bytes_fp32"] / (spmv_ms * 1e-3) / 1e9
    achieved_fmt = info["spmv_bytes_fp32"] / (spmv_ms * 1e-3) / 1e9
    n64 = sum(i["n_spmv_timed"] for i in inf_fp64_t)
    spmv64_ms = sum(i["t_spmv_ms"] for i in inf_fp64_t) / max(n64, 1)
    achieved64 = info["spmv_alg_bytes_fp64"] / (spmv64_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    timed_shape = mixed_t.info["spmv_shape_fp32"]
    traffic = profiled_traffic(SPMV_SOURCES, f"spmv_fp32_{args.workload}.md", timed_shape)
    its_fp64 = inf_fp64[-1]["iterations"]
    fp64_tf = optional(lambda: fp64_peak_tflops(dev))
    cpu, oracle_all, one = None, None, None
    if not args.no_cpu_baseline and world == 1:
        one = oracle_timing(args.workload, 1)
        cpu = {"value": one["ms"], "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"one full FP64 oracle solve to 1e-8 ({one['iterations']} iterations, "
                         f"1 thread), set-up ({one['setup_ms']:.0f} ms) excluded"}
        nc = host_cores()
        oracle_all = optional(lambda: oracle_timing(args.workload, nc))
        if isinstance(oracle_all, dict) and "ms" in oracle_all:
            oracle_all["cores"] = nc
    out = {
        "metric": METRIC, "value": t_mixed, "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_mixed,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 PCG / f64 residual replacement", "data": "synthetic",
        "config": config_dict(P, info["k"], args.workload),
        "fp64_ms": t_fp64, "speedup_mixed_vs_fp64": t_fp64 / t_mixed,
        "iterations_mixed": inf_mixed[-1]["iterations"],
        "outer_cycles_mixed": inf_mixed[-1]["outer_cycles"], "iterations_fp64": its_fp64,
        "iterations_oracle": one["iterations"] if one else None,
        "mixed_coarse_fp64": {"ms": max_over_ranks(pg, float(np.mean(ms_c64)), dev),
                              "iterations": inf_c64[-1]["iterations"],
                              "outer_cycles": inf_c64[-1]["outer_cycles"],
                              "rel_res_true": max(i["rel_res_true"] for i in inf_c64),
                              "note": "E^-1 applied in FP64 inside the FP32 iteration"},
        "graph": optional(graph_row),
        "iteration_gbs": optional(iteration_gbs),
        "rel_res_true_mixed": res_true, "rel_res_true_fp64": inf_fp64[-1]["rel_res_true"],
        "setup_ms": info["t_setup_ms"],
        "setup_phases_ms": {k: round(v, 1) for k, v in info["t_setup_phase_ms"].items()},
        "autotune": {"fp32_shape": info["spmv_shape_fp32"], "fp64_shape": fp64.info["spmv_shape_fp64"],
                     "fp32_shape_us": [round(t, 1) for t in info["spmv_shape_us_fp32"] if t >= 0],
                     "fp64_shape_us": [round(t, 1) for t in fp64.info["spmv_shape_us_fp64"]
                                       if t >= 0],
                     "timed_shape_fp32": mixed_t.info["spmv_shape_fp32"],
                     "shapes": "FP32 (steps/stage, stages, blocks/SM): (2,3,3) (1,4,4) (2,4,2) "
                               "(1,6,3) (3,3,2), lean kernel (2,3,3) (1,6,3) (2,2,4); "
                               "FP64: (1,3,3) (1,4,2) (2,2,2) (1,2,4)"},
        "spmv_fp32_gbs": achieved, "spmv_fp64_gbs": achieved64,
        "kernel_us_per_iteration": phases,
        "batched_load_cases": batch,
        "forward_backward": fwd_bwd,
        "propagation_sweep": sweep,
        "propagation_sequence": sequence,
        "subdomain_blocks": blocks_row,
        "iterations_vs_n": trend,
        "roofline": {"bound": "hbm", "kernel": spmv_kernel_name(timed_shape),
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": traffic, "algorithmic_bytes": info["spmv_alg_bytes_fp32"],
                     "format_bytes": info["spmv_bytes_fp32"], "achieved_format": achieved_fmt,
                     "avg_launch_ms": spmv_ms},
        "roofline_fp64_spmv": {"bound": "alu", "kernel": "k_spmv<double> (FP64 SpMV)",
                               "flops": 2 * info["nnz"], "avg_launch_ms": spmv64_ms,
                               "achieved_tflops": 2 * info["nnz"] / (spmv64_ms * 1e-3) / 1e12,
                               "peak_tflops": fp64_tf if isinstance(fp64_tf, float) else None,
                               "peak_source": "measured: cuBLAS DGEMM 4096^3 in this run",
                               "gbs": achieved64},
        "oracle_all_cores": oracle_all,
        "e2e": {"value": t_e2e, "unit": "ms", "h2d_bytes_per_step": 8 * P.n,
                "d2h_bytes_per_step": 8 * P.n},
        "gpu_launches": int(sum(i["n_launches"] for i in inf_mixed)),
        "clocks": clk,
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    print(json.dumps(out))


def run_profile(args):
    """One solve bracketed by cudaProfilerStart/Stop (for ncu --profile-from-start off)."""
    import torch
    import xfem_inputs as X
    from paper_2111_09294_gb300 import Solver
    if args.profile in ("sweep", "sweep_fused"):
        # one propagation sweep of --sweep systems, 8 load cases each
        from paper_2111_09294_gb300 import sweep as S
        Ps = X.make_many(X.SWEEP[:max(args.sweep, 1)])
        ssol = S.make_solvers(Ps, max_batch=8)
        Fs = [torch.tensor(X.load_cases(Pi, 8, seed=100 + i), device="cuda")
              for i, Pi in enumerate(Ps)]
        Us = [torch.empty_like(Fi) for Fi in Fs]
        fused = args.profile == "sweep_fused"
        for _ in range(max(args.warmup, 1)):
            S.solve_systems(ssol, Fs, TOL, outs=Us, fused=fused)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        res = S.solve_systems(ssol, Fs, TOL, outs=Us, fused=fused)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        infos = [i for _, inf in res for i in inf]
        print(json.dumps({"profile": args.profile, "systems": len(Ps),
                          "iterations_max": max(i["iterations"] for i in infos),
                          "rel_res_true_max": max(i["rel_res_true"] for i in infos)}))
        return
    P = X.make(args.workload)
    if args.profile == "batch":
        # the batched solve of args.batch seeded load cases
        s = Solver.from_problem(P, precision="mixed", inner_tol=args.inner_tol,
                                max_batch=args.batch)
        F = torch.tensor(X.load_cases(P, args.batch, seed=0), device="cuda")
        U = torch.empty_like(F)
        for _ in range(max(args.warmup, 1)):
            s.solve_batch(F, tol=TOL, out=U)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        _, infos = s.solve_batch(F, tol=TOL, out=U)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        info = infos[0]
        info["iterations"] = max(i["iterations"] for i in infos)
    else:
        s = Solver.from_problem(P, precision=args.profile, inner_tol=args.inner_tol)
        f = torch.tensor(P.f, device="cuda")
        u = torch.empty_like(f)
        for _ in range(max(args.warmup, 1)):
            s.solve(f, tol=TOL, out=u)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        _, info = s.solve(f, tol=TOL, out=u)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    print(json.dumps({"profile": args.profile, "iterations": info["iterations"],
                      "outer_cycles": info["outer_cycles"], "launches": info["n_launches"],
                      "t_solve_ms": info["t_solve_ms"], "info": s.info}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--inner-tol", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=8,
                    help="load cases of the batched-solve measurement (0: skip)")
    ap.add_argument("--sample-iters", type=int, default=10)
    ap.add_argument("--sweep", type=int, default=16,
                    help="also solve this many systems of the 32^3 propagation sweep "
                         "(<= 16; 0: skip)")
    ap.add_argument("--oracle-solve", action="store_true",
                    help="internal: one timed FP64 oracle solve of --workload, printed as JSON "
                         "(run in a child process with a fixed BLAS thread count)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=1,
                    help="time every SpMV pipeline shape at set-up and keep the fastest (0: "
                         "default shape)")
    ap.add_argument("--chain-steps", type=int, default=0,
                    help="with --workload cube64_penny_lognormal: also time the compliance "
                         "over this many crack-front steps (u recomputed, not stored)")
    ap.add_argument("--trend", type=int, default=1,
                    help="also report iterations against n at a fixed subdomain size (0: skip)")
    ap.add_argument("--subdomain-blocks", type=int, default=1,
                    help="also time block Jacobi with one block per subdomain (0: skip)")
    ap.add_argument("--profile", choices=["mixed", "fp64", "batch", "sweep", "sweep_fused"],
                    default=None,
                    help="profiler capture: one solve of the given path between "
                         "cudaProfilerStart/Stop after warm-up, nothing else timed")
    args = ap.parse_args()
    if args.oracle_solve:
        print(json.dumps(oracle_full_solve(args.workload)))
        return
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
