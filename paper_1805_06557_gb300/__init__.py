"""GB300-native REXI time step for the rotating shallow-water equations
(Schreiber, Schaeffer & Loft, arXiv 1805.06557).

The compute path is the C-ABI library ``librexi.so`` (hand-written sm_103a CUDA) built from
``csrc/``; ``rexi`` is its thin ctypes binding.  Importing this package does not load the
library: ``paper_1805_06557_gb300.rexi`` does, and raises if it is missing.
"""
