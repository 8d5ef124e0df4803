"""GB300-native iterative Sherman-Morrison EnKF analysis (libenkf_ism + binding).

Importing this package does not load the CUDA library; ``enkf.load()`` (called
by every binding function) does, and raises if it is missing.
"""
__all__ = ["build", "enkf"]
