"""GB300-native recycling BiCG (RBiCG) for sequences of dual sparse systems.

Importing the package loads nothing native; `paper_1010_0762_gb300.rbicg` loads the CUDA
library (built by `paper_1010_0762_gb300.build`) and fails loudly if it is missing.
"""
__all__ = ["inputs"]
