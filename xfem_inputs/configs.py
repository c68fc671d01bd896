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

All use nu = 0.3, z = 0 clamped and unit tension on z = 1; E = 1 unless a
per-element modulus is given.
"""
import os
import pickle
import tempfile

import numpy as np

from .assemble import build_problem
from .cracks import PlanarEdgeCrack, TiltedEllipticalCrack, WarpedEdgeCrack, WarpedPennyCrack

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


def make(name, cache=True):
    """Build (or load from a per-user temp cache) the named workload."""
    cfg = CONFIGS[name]
    path = os.path.join(tempfile.gettempdir(), f"xfem_inputs_{name}_{_source_hash()}.pkl")
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
