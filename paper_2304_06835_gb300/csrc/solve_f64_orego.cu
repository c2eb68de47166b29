// Solve kernels for the Orego stiff test model in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_orego, Orego, double)
