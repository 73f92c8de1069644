"""FP64 CPU oracle of the RKHS-BA hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline
and ``--impl reference`` legs may import this package.
"""
from .rkhs_oracle import *  # noqa: F401,F403
from .rkhs_oracle import __all__  # noqa: F401
