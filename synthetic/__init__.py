"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package only *builds inputs*: real-space model tensors H(R_e), D(R_p),
g~(R_e, R_p), lattice data, Monkhorst-Pack point lists and initial occupations.
It holds none of the method's arithmetic (no Fourier sums, no diagonalisation,
no matrix-element rotation, no rates); those live separately in ``oracle/``
(CPU, FP64, test infrastructure) and in ``paper_2002_02045_gb300`` (CUDA).
"""
from .models import (  # noqa: F401
    Model,
    SEED_BASE,
    mp_grid,
    model_c1,
    model_c2,
    model_c3,
    model_batch_instance,
    model_sc_tight_binding,
    model_holstein,
    model_ladder,
    pulse_occupations,
)
