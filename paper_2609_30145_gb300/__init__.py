"""GB300-native (sm_103a) batched SED forward model and Gaussian log-likelihood.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/sed.h``); ``api`` is a thin binding over it.
"""
from .api import Context, Model, SedError, SedLogLike, Server, PREC  # noqa: F401
