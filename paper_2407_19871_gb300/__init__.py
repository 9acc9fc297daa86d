"""GB300-native TFHE gate bootstrapping and LocPIR circuits (arXiv 2407.19871).

The compute path is liblocpir.so (CUDA for sm_103a, C-ABI in include/locpir.h);
`locpir` is its thin ctypes binding.  Build the library with
`python -m paper_2407_19871_gb300.build`.
"""
from . import locpir  # noqa: F401
from .locpir import Context, LocpirError  # noqa: F401
