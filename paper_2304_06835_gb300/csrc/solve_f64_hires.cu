// Solve kernels for the Hires stiff test model in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_hires, Hires, double)
