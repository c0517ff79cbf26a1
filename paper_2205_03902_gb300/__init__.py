"""GB300-native hot path of inverse multislice ptychography (arXiv 2205.03902).

`msp` is the Python binding of the C ABI in `include/msp.h`; `build` compiles
the sm_103a library in-tree.
"""
from . import msp  # noqa: F401
