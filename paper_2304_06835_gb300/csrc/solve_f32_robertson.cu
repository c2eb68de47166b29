// Solve kernels for the Robertson model in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_robertson, Robertson, float)
