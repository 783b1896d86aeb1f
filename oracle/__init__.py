"""FP64 CPU oracle of the cascaded lattice Boltzmann method (Liu & He).

TEST INFRASTRUCTURE ONLY: the plain reference that the CUDA path is checked
against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
leg import it; the product package never does.  It shares no code with the CUDA
library.  See ``clb_oracle.c`` for the algorithm, its equation citations and the
readings taken where the paper is silent.
"""
from .oracle import (  # noqa: F401
    OracleParams,
    OracleSim,
    build_oracle,
    collide,
    feq,
    flow_sum_cs,
    gradient_cs,
    kmat,
    lattice,
    load,
    r_from_sigma,
    rates_kn,
    step_nodes,
    threads_used,
    tinv,
    tmat,
)
