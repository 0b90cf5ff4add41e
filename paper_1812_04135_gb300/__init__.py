"""GB300-native RSST finite-volume step (arXiv:1812.04135).

The compute path is the CUDA library ``librsst.so`` (C ABI declared in
include/rsst.h); ``rsst`` is its thin Python binding.  ``inputs`` builds the
seeded synthetic initial states.
"""
