"""CPU oracle for the LEC-QMC hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_2601_08552_gb300``.
"""
from .oracle import OracleSim, build_oracle, comb, philox4x32_10, NOBS, OBS_NAMES  # noqa: F401
from . import lattices  # noqa: F401
