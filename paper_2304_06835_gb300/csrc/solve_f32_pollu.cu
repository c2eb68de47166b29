// Solve kernels for the Pollu stiff test model in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_pollu, Pollu, float)
