"""CPU oracle of the Generals.io environment step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` load this package.  The CUDA library never imports it, links it
or calls it.  The rules live in ``generals_oracle.c`` (plain single-threaded
C, one cell at a time); this module only compiles that file and marshals
arguments through ctypes.
"""
from .orc import OracleEnv, OracleParams, build_oracle, oracle_lib, sm, key, draw  # noqa: F401
