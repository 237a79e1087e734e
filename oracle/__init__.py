"""FP64 CPU oracle for the multi-messenger Wiener filter (Huffenberger 2017).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm use it.  It shares no code with
the CUDA path; both take their inputs from ``paper_1704_00865_gb300.synth``.
"""

from .wf_oracle import *  # noqa: F401,F403
from . import fno_oracle  # noqa: F401
