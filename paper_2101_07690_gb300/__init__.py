"""GB300 frequent subgraph mining with two-vertex exploration.

The mining itself lives in the CUDA library built from ``csrc/`` (C ABI: include/fsm.h);
``fsm`` is its Python binding.  Importing this package does not load the library: call
``paper_2101_07690_gb300.fsm.load()`` (or use ``fsm.Graph``), which raises if it is missing.
"""
from . import fsm  # noqa: F401

__all__ = ["fsm"]
