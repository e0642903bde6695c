"""CPU oracle of the differentiable light-stage renderer (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never links it.
"""
from .oracle import (Oracle, OracleConfig, default_config, build_oracle,  # noqa: F401
                     ORACLE_SO)
