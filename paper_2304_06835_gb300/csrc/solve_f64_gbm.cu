// Solve kernels for the GBM model in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_gbm, GBM, double)
