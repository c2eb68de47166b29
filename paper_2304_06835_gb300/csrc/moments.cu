// moments.cu -- ensemble sums for moment estimation (the post-solve exchange of a sharded SDE
// ensemble: each rank reduces its own trajectories, the ranks add their sums).
//
// Pass 1: ENS_MOMENTS_BLOCKS blocks (4 per SM of a GB300) stride over the trajectories and
// add, per component, x and x^2 in FP64 over the trajectories whose status is OK (all, without
// a status array); each block reduces its threads in a fixed order (a shuffle tree per warp,
// then warp 0 over the warp sums) and writes its partial sums to the caller's scratch.
// Pass 2: one block adds the partials of every entry in a fixed order.  The result does not
// depend on timing, and the reads run at HBM speed (a single block left them latency-bound).
#include "ens_internal.h"

namespace ens {
namespace {

constexpr int kMomThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // sh is reused across calls
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  v = lane < (int)(blockDim.x >> 5) && warp == 0 ? sh[lane] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;  // valid in thread 0
}

// partial[b * (2D + 1) + e], e < 2D + 1: block b's sums of x_j (e = j), x_j^2 (e = D + j), n
template <class T>
__global__ void __launch_bounds__(kMomThreads)
    k_moments_partial(long long N, int D, int layout, int S, int slot, const T* out,
                      const signed char* status, double* partial) {
  __shared__ double sh[32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  double* mine = partial + (long long)blockIdx.x * (2 * D + 1);
  for (int j = 0; j < D; ++j) {
    double s1 = 0.0, s2 = 0.0, c = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
      if (status && status[i] != 0) continue;
      const long long k = layout == ENS_LAYOUT_SOA ? ((long long)slot * D + j) * N + i
                                                   : (i * S + slot) * (long long)D + j;
      const double x = (double)out[k];
      s1 += x;
      s2 = fma(x, x, s2);
      c += 1.0;
    }
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (j == 0) c = block_sum(c, sh);
    if (threadIdx.x == 0) {
      mine[j] = s1;
      mine[D + j] = s2;
      if (j == 0) mine[2 * D] = c;
    }
  }
}

__global__ void __launch_bounds__(kMomThreads)
    k_moments_final(int E, int G, const double* partial, double* sums) {
  __shared__ double sh[32];
  for (int e = 0; e < E; ++e) {
    double v = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) v += partial[(long long)b * E + e];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) sums[e] = v;
  }
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" int ens_moments(long long N, int D, int dtype, int layout, int S, int slot,
                           const void* out, const signed char* status, double* scratch,
                           double* sums, void* cuda_stream) {
  if (N < 0 || D < 1 || S < 1) return set_last_error(ENS_EINVAL, "bad sizes");
  if (slot < 0 || slot >= S) return set_last_error(ENS_EINVAL, "slot out of range");
  if (dtype != ENS_F32 && dtype != ENS_F64) return set_last_error(ENS_EINVAL, "unknown dtype");
  if (layout != ENS_LAYOUT_SOA && layout != ENS_LAYOUT_ROWMAJOR)
    return set_last_error(ENS_EINVAL, "unknown layout");
  if (!sums || !scratch || (N > 0 && !out)) return set_last_error(ENS_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int G = ENS_MOMENTS_BLOCKS;
  if (dtype == ENS_F32)
    k_moments_partial<float><<<G, kMomThreads, 0, s>>>(
        N, D, layout, S, slot, static_cast<const float*>(out), status, scratch);
  else
    k_moments_partial<double><<<G, kMomThreads, 0, s>>>(
        N, D, layout, S, slot, static_cast<const double*>(out), status, scratch);
  k_moments_final<<<1, kMomThreads, 0, s>>>(2 * D + 1, G, scratch, sums);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ENS_OK : set_last_error(ENS_ECUDA, cudaGetErrorString(e));
}
