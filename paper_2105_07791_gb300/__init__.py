"""GB300-native nested-dissection preconditioner with dense and HSS-compressed fronts.

The compute path lives in the CUDA library ``lib/libndhss.so`` (C ABI in
``include/ndhss.h``); ``ndhss`` is its thin Python binding.
"""
from . import build  # noqa: F401
