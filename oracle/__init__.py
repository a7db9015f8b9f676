"""Test infrastructure: the FP64 CPU oracle for the pressure projection.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path (the CUDA library and its
Python binding) never imports, calls or links anything here, and this package
imports nothing from the product.
"""
from .pressure_oracle import *  # noqa: F401,F403
