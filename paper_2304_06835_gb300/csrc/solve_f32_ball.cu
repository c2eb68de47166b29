// Solve kernels for the bouncing ball (events) in float.
#include "solve_impl.cuh"
ENS_INSTANTIATE_MODEL(dispatch_f32_ball, Ball, float)
