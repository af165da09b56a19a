"""CPU FP64 oracle for the multibody MFS scattering solve.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
links this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library; the only module both sides draw from is ``mbs_inputs`` (seeded
geometry and incident fields, no solver arithmetic).

Parity status of each function is stated in ``mbs_oracle``'s header.
"""
from .mbs_oracle import *  # noqa: F401,F403
