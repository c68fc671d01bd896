"""GB300-native adapted deflated CG (A-DEF2 + block Jacobi) for XFEM crack systems."""
from .solver import Elements, Pattern, Solver
from ._lib import XdcgError, load

__all__ = ["Elements", "Pattern", "Solver", "XdcgError", "load"]
