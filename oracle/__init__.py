"""FP64 reference integrator (the oracle) for coupled linear oscillators.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain single-threaded C program
(``cho_oracle.c``) plus this ctypes wrapper.  Only the tests, the smoke check
and the CPU-baseline leg of the benchmark may import it; the library under
``paper_1702_02207_gb300`` never does, and the oracle imports nothing from it.
"""
from .oracle import (  # noqa: F401
    build,
    load,
    rk4_chain,
    rk4_chain_ext,
    rk4_dense,
    energy_chain,
    energy_dense,
)
