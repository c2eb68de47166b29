// Solve kernels for the GBM model in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_gbm, GBM, float)
