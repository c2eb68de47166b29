// Solve kernels for the Pollu stiff test model in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_pollu, Pollu, double)
