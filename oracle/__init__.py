"""CPU oracle of the third-order DUGKS step (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
reference arm of ``bench.py`` may import this package.  The product path
(``paper_1709_05458_gb300``) shares no code with it and never imports it.

Parity status of each function is listed in ``dugks_oracle.py``; every
function here is pinned by a test under ``tests/test_oracle_*.py``.
"""
from . import dugks_oracle, velocity_sets  # noqa: F401
