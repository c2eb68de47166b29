// Solve kernels for the Orego stiff test model in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_orego, Orego, float)
