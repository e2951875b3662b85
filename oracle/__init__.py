"""CPU oracle for the NURSD operator -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 NumPy statement of what the operator computes, written
from the paper (arXiv 2501.05244) and pinned by CPU tests against closed forms,
brute force and special cases.  It shares no code with the CUDA library and
does not import it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the product path never does.
"""
from .nursd_oracle import *  # noqa: F401,F403
