// Solve kernels for the sigma-factor CRN SDE in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_crn, CRN, double)
