"""FP64 CPU oracle of Simpler balanced splitting and ROK4E -- TEST INFRASTRUCTURE.

A plain, slow, obviously-checkable restatement of the method in numpy, used by
``tests/``, by ``__graft_entry__.smoke()`` and by the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``.  It shares no code with the CUDA
library (``paper_1712_00953_gb300``) and neither imports the other; only the
seeded input generators in ``synth`` serve both.

Modules:
  kinetics   constant-pressure reactor RHS f(u) and its dense Jacobian
  rok4e      Arnoldi, one ROK4E attempt, Algorithm 1 with PI control
  splitting  Strang / balanced / Simpler steps, scalar recurrences, 1-D case
  c_oracle   the same method compiled from C (oracle/c/), pinned against the
             modules above; for long horizons and the timed CPU baseline
"""

from . import kinetics, rok4e, splitting  # noqa: F401
