"""GB300-native decomposed-kernel (FAGP) Gaussian process.

Fit and predict the posterior of Sec. 2.2 of arXiv 2403.12797 with the SE
kernel's Hermite eigenfunctions taken as a tensor product over the input
dimensions (Sec. 2.3). All computation runs in the CUDA kernels of
``libgpfagp.so`` (C ABI in ``include/gpfagp.h``); this package only
marshals arguments.
"""
from ._lib import (GPError, Model, fit, fit_batch, fit_plain, fit_predict, gram, lib, predict_batch,  # noqa: F401
                   strerror, version)
