"""GB300-native TPU-KNN search path (arXiv 2206.14286).

The search runs in the CUDA library ``libtpuknn.so`` built from ``csrc/``;
this package is its thin Python binding (argument marshalling only).
"""
__version__ = "0.1.0"
