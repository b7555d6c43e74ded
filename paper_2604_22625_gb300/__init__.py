"""GB300-native solver for the FlashFolio portfolio models (single- and multi-period).

The compute path is the CUDA library ``libflashfolio.so`` (C ABI in
``include/flashfolio.h``); ``api`` moves problems to the GPU with PyTorch and
calls it.  Importing the package does not load the library; ``api`` and
``_lib`` load it on first use and raise if it is missing.
"""
__all__ = ["api", "autograd", "build", "replicas", "synthetic", "tune"]
