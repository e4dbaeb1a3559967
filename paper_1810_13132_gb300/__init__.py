"""GB300 (sm_103a) implementation of VBDR, sliding-window host-cardinality
estimation with shared HyperLogLog bit distance recorders (arXiv 1810.13132).

The method runs in the CUDA library ``libvbdr.so`` behind the C ABI declared in
``include/vbdr.h``; ``Vbdr`` is its thin Python binding.
"""
from .vbdr import (CompactNet, Config, Mlp, Plan, Server, Vbdr, VbdrError,  # noqa: F401
                   exported_symbols, live_features, load)
