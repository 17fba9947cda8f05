"""GB300-native FFT-based bandwidth selection for multivariate KDE.

Implements the hot path of Gramacki & Gramacki (arXiv 1511.07482): linear
binning, sampled Gaussian-derivative kernel grids for full bandwidth
matrices, zero-padded d-dimensional FFTs and the spectral multiply-and-
reduce, for psi_r, LSCV, SCV and plug-in objectives with gradients.  The
compute runs in libkdefft.so (hand-written CUDA for sm_103a) behind the C ABI
of include/kdefft.h; this package is a thin binding.
"""
from ._lib import (  # noqa: F401
    Context, Dataset, KdefftError, default_opts, load,
    L_AUTO, L_PAPER, L_WIDEST, L_FULL, P_MINIMAL, P_PAPER, P_PAPER_FULL, P_FIXED,
    FP32, FP64, BIN_LINEAR, BIN_SIMPLE, OUTSIDE_ERROR, OUTSIDE_DROP, LSCV, SCV, PI,
    DT_F32, DT_F64, DT_I32, EXPORTS, ENGINE_AUTO, ENGINE_MULTIPASS, ENGINE_HOST_SELECT, ENGINE_FFT,
)
