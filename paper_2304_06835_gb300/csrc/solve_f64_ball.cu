// Solve kernels for the bouncing ball (events) in double.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f64_ball, Ball, double)
