"""Seeded synthetic inputs: vector recipes (``gen``) and the input-PG builder (``pgbuild``).

Serves both the CPU oracle and the CUDA path; holds none of the merge arithmetic.
"""
from . import gen  # noqa: F401
from .pgbuild import build_pg, build_all  # noqa: F401
