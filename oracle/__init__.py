"""FP64 CPU oracle for the e-ph hot path (TEST INFRASTRUCTURE ONLY).

This package is the plain, slow, obviously correct statement of what the
GPU path computes, written from the equations of the Perturbo paper
(arXiv 2002.02045).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product package never imports it and shares no code, constants or
helpers with it; both sides only consume inputs built by ``synthetic/``.

Parity status of every function is listed in the module docstring of
``oracle.eph``.
"""
from . import eph  # noqa: F401
