// Solve kernels for the Lorenz model in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_lorenz, Lorenz, float)
