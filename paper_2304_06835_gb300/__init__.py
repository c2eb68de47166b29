"""GB300-native ensemble ODE/SDE solver (arXiv 2304.06835's data-parallel hot path).

The compute path is libens.so (hand-written CUDA for sm_103a behind a C ABI, include/ens.h);
this package only marshals torch tensors into it.
"""
from ._lib import EnsError, lib  # noqa: F401
from .solver import (EnsembleBatch, EnsembleSolver, combine_moments,  # noqa: F401
                     ensemble_moments, gather_moments, make_opts, merge_moments, normals,
                     philox_words)
from .autograd import solve_fixed  # noqa: F401
from .shard import shard_plan, solve_sharded  # noqa: F401
from .surrogate import GatedSurrogate, SurrogateMLP  # noqa: F401

__all__ = ["EnsembleBatch", "EnsembleSolver", "EnsError", "combine_moments", "ensemble_moments",
           "gather_moments", "merge_moments", "make_opts", "normals", "philox_words", "lib", "shard_plan", "solve_sharded",
           "solve_fixed", "SurrogateMLP", "GatedSurrogate"]
