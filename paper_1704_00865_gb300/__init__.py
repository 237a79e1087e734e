"""GB300-native multi-messenger Wiener filter (Huffenberger 2017, arXiv:1704.00865).

The solver itself lives in a CUDA shared library (``libwf.so``, C ABI declared
in ``include/wf.h``); :mod:`paper_1704_00865_gb300.wf` is the thin ctypes
binding and :mod:`paper_1704_00865_gb300.synth` makes seeded synthetic inputs.
"""

__all__ = ["synth", "wf"]
