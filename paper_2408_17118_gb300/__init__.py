"""GB300-native batched kurtosis fixed-point iteration of the ordering ICA (arXiv 2408.17118).

The computation lives in ``libica.so`` (C ABI, ``include/ica.h``); ``ica`` is its Python
binding. Importing this package does not load CUDA; the binding loads the library on first
use and raises if it has not been built.
"""
from ._lib import ICA_BF16, ICA_FP32, ICA_PLAIN_FP32, LIB_PATH  # noqa: F401

__all__ = ["ICA_BF16", "ICA_FP32", "ICA_PLAIN_FP32", "LIB_PATH"]
