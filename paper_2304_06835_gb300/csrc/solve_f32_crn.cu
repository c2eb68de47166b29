// Solve kernels for the sigma-factor CRN SDE in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_crn, CRN, float)
