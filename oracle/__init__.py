"""CPU float64 oracle for contractions of cyclic-group-symmetric tensors.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package.  The product path (the CUDA library and its
Python binding) never imports it, and this package never imports the
product path: the two share no code.

Parity status: every routine here is pinned by ``tests/test_oracle_*.py``
to something other than itself (brute force on tiny inputs, closed-form
counts, textbook special cases, invariants fixed by the paper's proof).
"""
from .symoracle import *  # noqa: F401,F403
