"""GB300-native random-forest fit / predict / device selection for AIWC features.

Importing the package loads nothing: ``paper_1811_00156_gb300.aiwcrf`` loads the CUDA library
and fails loudly when it is missing.
"""
