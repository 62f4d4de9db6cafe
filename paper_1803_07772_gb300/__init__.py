"""GB300-native solver for energy-efficient resource allocation in PD-NOMA
H-CRANs (arXiv 1803.07772): Dinkelbach around SCALE + Lagrangian dual
iterations, as hand-written CUDA for sm_103a behind a small C ABI.
"""
from .hcran import HcranError, Solver, Tol, load, make_tol  # noqa: F401
