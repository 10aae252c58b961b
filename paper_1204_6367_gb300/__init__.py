"""GB300-native gDRR: Monte Carlo x-ray projection (arXiv:1204.6367).

Importing the package is light: the CUDA library binding is loaded by
``paper_1204_6367_gb300.gdrr`` on first use and fails loudly when the
compiled library is missing.
"""
__all__ = ["inputs", "gdrr"]
