// Solve kernels for the Lorenz model in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_lorenz, Lorenz, double)
