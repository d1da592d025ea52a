"""GB300-native pixel track seeding and broken-line fitting (arXiv 2008.13461).

The compute path lives in the CUDA library libpt_gb300.so (C ABI in
include/pt.h), loaded through ``paper_2008_13461_gb300._lib``; ``Pipeline``
in ``paper_2008_13461_gb300.pipeline`` is the user-facing entry point.
Importing this package loads nothing; the library is loaded on first use.
"""
__all__ = ["build", "pipeline"]
