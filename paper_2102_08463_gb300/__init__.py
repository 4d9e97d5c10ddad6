"""GB300-native 2D/3D type 1 and type 2 nonuniform FFT (arXiv 2102.08463).

The compute path is the C-ABI shared library built from ``csrc/`` (CUDA for
sm_103a plus cuFFT for the fine-grid FFT).  ``binding`` wraps it with ctypes;
importing this package does not load the library until it is first used.
"""
__all__ = ["binding", "workloads"]
