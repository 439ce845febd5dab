"""GB300-native belief-propagation polar decoder (arXiv 1505.04979).

The decoder itself lives in the CUDA library ``csrc/`` builds
(``libpolarbp.so``); :mod:`paper_1505_04979_gb300.binding` marshals arguments
to its C ABI.  Importing this package loads nothing: the library is loaded on
first use, and the binding raises if it is missing.
"""

__all__ = ["binding", "inputs", "build"]
