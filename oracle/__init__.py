"""CPU FP64 oracle of the RSST finite-volume step.

Test infrastructure only: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the product path.
"""
from . import rsst_oracle, adjoint, riemann_exact  # noqa: F401
