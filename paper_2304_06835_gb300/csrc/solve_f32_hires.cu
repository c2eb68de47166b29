// Solve kernels for the Hires stiff test model in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_hires, Hires, float)
