"""B300-native sliced pairwise contraction of quantum-circuit tensor networks.

The compute path is libjet.so (CUDA kernels for sm_103a behind the C ABI of
include/jet.h); `jet` is its ctypes binding and `autograd` its
torch.autograd.Function wrapper.
"""
from .jet import (Network, JetError, default_options, from_network, lib, PREC, EXPORTS,  # noqa: F401
                  JET_OK, JET_EINVAL, JET_ENOMEM, JET_ECUDA, JET_ETIMEOUT, JET_ESTATE)
