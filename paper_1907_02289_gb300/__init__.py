"""GB300 (sm_103a) group-shared Barnes-Hut tree force evaluation.

The compute path lives in the CUDA library ``libbh.so`` (sources in ``csrc/``,
C ABI declared in ``include/bh.h``); ``bh`` is its thin ctypes binding.
Importing this package does not load the library; ``bh.load()`` does, and
fails loudly when it is missing.
"""
__all__ = ["bh", "synth"]
