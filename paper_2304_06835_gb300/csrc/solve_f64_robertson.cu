// Solve kernels for the Robertson model in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_robertson, Robertson, double)
