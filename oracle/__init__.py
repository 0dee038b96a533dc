"""FP64 CPU oracle of the N-phase conservative Allen-Cahn lattice Boltzmann
method (arXiv 2306.06983).  Test infrastructure only: imported by the tests,
the smoke check and the benchmark's CPU-baseline leg, never by the library."""

from .oracle import OracleSim, build_oracle, oracle_lib, oracle_lib_fp32, params_struct  # noqa: F401
