"""GB300-native Ito-KMC streamer step (arXiv 2307.01797).

The compute path is the C-ABI library ``libitokmc.so`` built from ``csrc/``
(hand-written sm_103a CUDA); ``itokmc`` is its thin ctypes binding and
``synth`` the seeded synthetic-input generator.
"""
