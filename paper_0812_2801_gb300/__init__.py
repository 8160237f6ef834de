"""GB300-native modified-Ehrenfest TDDFT molecular dynamics (arXiv:0812.2801).

Importing the package loads nothing compiled; ``paper_0812_2801_gb300.emd``
loads the CUDA library ``libemd.so`` on first use and raises if it is missing.
"""
__all__ = ["inputs", "emd", "adjoint", "autotune", "precision", "vibrations"]
