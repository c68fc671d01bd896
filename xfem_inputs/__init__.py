"""Seeded synthetic XFEM crack systems: the inputs shared by the oracle and the GPU harness."""
from .assemble import (KIND_HEAVISIDE, KIND_STD, KIND_TIP, Problem, build_problem, by_subdomain,
                       to_dense)
from .configs import (CONFIGS, STEPS64, SWEEP, SWEEP_RADII, TREND, TREND_M, make,
                      make_many)
from .elements import element_data
from .loads import face_weights, load_cases, tractions
