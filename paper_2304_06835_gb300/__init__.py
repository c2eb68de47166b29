"""GB300-native ensemble ODE/SDE solver (arXiv 2304.06835's data-parallel hot path).

The compute path is libens.so (hand-written CUDA for sm_103a behind a C ABI, include/ens.h);
this package only marshals torch tensors into it.
"""
from ._lib import EnsError, lib  # noqa: F401
from .solver import (EnsembleBatch, EnsembleSolver, combine_moments, ensemble_sums,  # noqa: F401
                     make_opts, normals, philox_words)
from .autograd import solve_fixed  # noqa: F401
from .surrogate import GatedSurrogate, SurrogateMLP  # noqa: F401

__all__ = ["EnsembleBatch", "EnsembleSolver", "EnsError", "combine_moments", "ensemble_sums",
           "make_opts", "normals", "philox_words", "lib",
           "solve_fixed", "SurrogateMLP", "GatedSurrogate"]
