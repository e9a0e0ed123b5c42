"""GB300-native batched first-person raycasting environments (JAXenstein's hot path).

The compute path lives in ``csrc/`` (hand-written CUDA for sm_103a behind a C
ABI, declared in ``include/jx.h``); ``jx`` is the thin ctypes binding over it.
``inputs`` holds the seeded workload presets and random action streams.
Importing this package does not load the CUDA library; ``jx`` does, and it
raises if the library is missing.
"""

__all__ = ["inputs", "jx"]
