"""The synthetic workloads, named by mesh size and crack.

* cube8_edge:        8^3 hexes, planar edge crack phi = z - 0.5, psi = x - 0.45,
                     r_e = 0.15, 2^3 boxes.
* cube24_ellipse:    24^3 hexes, inclined elliptical crack (semi-axes 0.30 /
                     0.20, centre (0.5, 0.5, 0.5), tilted 30 deg about x,
                     warped by 0.03 sin(2 pi x)), r_e = 0.08, 4^3 boxes.
* cube48_two_cracks: 48^3 hexes, warped penny (radius 0.2 centred over
                     (0.5, 0.5) at z = 0.3) and warped edge crack (z = 0.7,
                     depth 0.25 from x = 0), warp 0.02 sin(2 pi y) cos(2 pi x),
                     r_e = 0.05, 8^3 boxes.
* cube64_penny_lognormal: 64^3 hexes, warped penny (radius 0.3 centred at
                     (0.5, 0.5, 0.5), the same warp), r_e = 0.05, 8^3 boxes,
                     per-element Young's modulus log-normal (mu 0, sigma 0.3,
                     seed 0): the differentiable-solve workload.
* cube64_penny_lognormal_step1 .. _step3: the same with the penny's radius
                     0.32, 0.34, 0.36: four crack-front positions for a
                     differentiable solve over propagation steps.
* trend12 .. trend48: the cube24_ellipse crack at 12^3 .. 48^3 hexes, boxes
                     of 6^3 hexes, r_e = 2 h: iterations against n at a
                     fixed subdomain size.
* cube32_sweep_00 .. cube32_sweep_15: 32^3 hexes, an inclined penny
                     (centre (0.5, 0.5, 0.5), tilted 30 deg about x, no warp)
                     whose radius grows linearly from 0.15 to 0.35 over the 16
                     systems, r_e = 0.07, 8^3 boxes: successive crack-front
                     positions of a propagation sweep (the radii are
                     prescribed; no growth law is computed).

All use nu = 0.3, z = 0 clamped and unit tension on z = 1; E = 1 unless a
per-element modulus is given.
"""
import os
import pickle
import tempfile

import numpy as np

from .assemble import build_problem
from .cracks import PlanarEdgeCrack, TiltedEllipticalCrack, WarpedEdgeCrack, WarpedPennyCrack

SWEEP_RADII = np.linspace(0.15, 0.35, 16)
SWEEP = [f"cube32_sweep_{i:02d}" for i in range(len(SWEEP_RADII))]

CONFIGS = {
    "cube8_edge": dict(m=8, n_box=2,
                       cracks=lambda: [PlanarEdgeCrack(0.5, 0.45, 0.15)]),
    "cube24_ellipse": dict(m=24, n_box=4,
                           cracks=lambda: [TiltedEllipticalCrack((0.5, 0.5, 0.5), 0.30, 0.20,
                                                                 np.deg2rad(30.0), 0.03, 0.08)]),
    "cube48_two_cracks": dict(m=48, n_box=8,
                              cracks=lambda: [WarpedPennyCrack((0.5, 0.5, 0.3), 0.2, 0.02, 0.05),
                                              WarpedEdgeCrack(0.7, 0.25, 0.02, 0.05)]),
    "cube64_penny_lognormal": dict(m=64, n_box=8,
                                   cracks=lambda: [WarpedPennyCrack((0.5, 0.5, 0.5), 0.3, 0.02,
                                                                    0.05)],
                                   young=lambda m: np.random.default_rng(0).lognormal(
                                       0.0, 0.3, m ** 3)),
}
# iterations against system size at a fixed subdomain size (Section 4.1's
# scalability study): the 24^3 case's crack at m = 12 .. 48 hexes per axis,
# boxes of 6^3 hexes (n / n_sd about 650-730), tip radius 2 h
TREND_M = (12, 24, 36, 48)
TREND = [f"trend{m}" for m in TREND_M]
for _m in TREND_M:
    CONFIGS[f"trend{_m}"] = dict(m=_m, n_box=_m // 6,
                                 cracks=lambda m=_m: [TiltedEllipticalCrack(
                                     (0.5, 0.5, 0.5), 0.30, 0.20, np.deg2rad(30.0), 0.03,
                                     2.0 / m)])
# four successive crack-front positions of the 64^3 log-normal workload (the
# penny grows by 0.02 a step; prescribed, no growth law), same moduli
STEPS64 = ["cube64_penny_lognormal"] + [f"cube64_penny_lognormal_step{s}" for s in (1, 2, 3)]
for _s in (1, 2, 3):
    CONFIGS[f"cube64_penny_lognormal_step{_s}"] = dict(
        m=64, n_box=8,
        cracks=lambda s=_s: [WarpedPennyCrack((0.5, 0.5, 0.5), 0.3 + 0.02 * s, 0.02, 0.05)],
        young=CONFIGS["cube64_penny_lognormal"]["young"])
for _name, _r in zip(SWEEP, SWEEP_RADII):
    CONFIGS[_name] = dict(m=32, n_box=8,
                          cracks=lambda r=float(_r): [TiltedEllipticalCrack(
                              (0.5, 0.5, 0.5), r, r, np.deg2rad(30.0), 0.0, 0.07)])


def _source_hash():
    """Hash of this package's sources: a cached problem is reused only while
    the generator is unchanged."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.dirname(os.path.abspath(__file__))
    for f in sorted(os.listdir(d)):
        if f.endswith(".py"):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:12]


def _cache_path(name):
    return os.path.join(tempfile.gettempdir(), f"xfem_inputs_{name}_{_source_hash()}.pkl")


def make(name, cache=True):
    """Build (or load from a per-user temp cache) the named workload."""
    cfg = CONFIGS[name]
    path = _cache_path(name)
    if cache and os.path.exists(path):
        with open(path, "rb") as fh:
            return pickle.load(fh)
    young = cfg["young"](cfg["m"]) if "young" in cfg else None
    P = build_problem(cfg["m"], cfg["cracks"](), cfg["n_box"], young=young)
    P.name = name
    if cache:
        tmp = path + f".{os.getpid()}"
        with open(tmp, "wb") as fh:
            pickle.dump(P, fh, protocol=pickle.HIGHEST_PROTOCOL)
        os.replace(tmp, path)
    return P


def _make_cached(name):
    make(name)
    return name


def make_many(names, workers=8):
    """make() for several workloads, the missing ones built in parallel
    worker processes (spawned, so a parent that already uses CUDA is safe)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    todo = [n for n in names if not os.path.exists(_cache_path(n))]
    if len(todo) > 1 and workers > 1:
        with cf.ProcessPoolExecutor(min(workers, len(todo)),
                                    mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_make_cached, todo))
    return [make(n) for n in names]
