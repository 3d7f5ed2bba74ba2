"""GB300-native FFT multichannel interpolation (Cheng & Kou, arXiv 1802.10291).

Importing the package loads nothing: the CUDA library is opened on first use
by :mod:`paper_1802_10291_gb300.mci`, which raises when it is missing.
"""
__all__ = ["mci", "synth"]
