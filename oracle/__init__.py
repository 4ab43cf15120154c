"""FP64 CPU oracle of the DIGS hot path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` / ``--impl reference``
legs may import this package.  It shares no code with the CUDA path.
"""
from . import digs_oracle  # noqa: F401
