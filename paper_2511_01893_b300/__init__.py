"""B300-native laminographic operator L / L^H and fused ADMM-TV.

The compute path is the CUDA library ``liblamino.so`` built from ``csrc/``
and reached through the C ABI declared in ``include/lamino.h``; ``lamino``
is the thin ctypes binding.  Importing this package loads nothing; the
library is loaded on first use and a missing library raises.
"""
