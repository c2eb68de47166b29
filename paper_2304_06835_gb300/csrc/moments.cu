// moments.cu -- ensemble moments for Monte Carlo estimation (the post-solve exchange of a
// sharded SDE ensemble: each rank reduces its own trajectories, the ranks merge the results).
//
// Per component the reduction carries (n, mean, M2), M2 = sum of squared deviations from the
// mean, and joins two groups with the pairwise update of Chan, Golub and LeVeque (1979):
//   n = n_a + n_b,  delta = mean_b - mean_a,  mean = mean_a + delta n_b / n,
//   M2 = M2_a + M2_b + delta^2 n_a n_b / n.
// Raw power sums (sum x, sum x^2) lose the variance to cancellation when |mean| >> std (a
// species count far from zero); the merged form does not.
// Pass 1: ENS_MOMENTS_BLOCKS blocks (4 per SM of a GB300) stride over the trajectories.  A
// thread accumulates sums of x - K and (x - K)^2 about K, the first value it reads, which
// lies within the spread of its values, then turns them into its own (n, mean, M2); threads
// merge by a shuffle tree per warp, then warp 0 over the warp results, and each block writes
// its partial to the caller's scratch.  Pass 2: one block merges the partials, each thread a
// fixed set of blocks in order, then the same tree.  The result does not depend on timing.
#include <cmath>

#include "ens_internal.h"

namespace ens {
namespace {

constexpr int kMomThreads = 256;

struct Mom {
  double n, mean, m2;
};

__device__ __forceinline__ Mom merge(const Mom& a, const Mom& b) {
  const double n = a.n + b.n;
  if (n == 0.0) return Mom{0.0, 0.0, 0.0};
  const double d = b.mean - a.mean, fb = b.n / n;
  return Mom{n, fma(d, fb, a.mean), fma(d * d * a.n, fb, a.m2 + b.m2)};
}

__device__ __forceinline__ Mom shfl_down(const Mom& v, int o) {
  return Mom{__shfl_down_sync(0xffffffffu, v.n, o), __shfl_down_sync(0xffffffffu, v.mean, o),
             __shfl_down_sync(0xffffffffu, v.m2, o)};
}

// merge over the block's threads in a fixed order; valid in thread 0
__device__ __forceinline__ Mom block_merge(Mom v, Mom* sh) {
  for (int o = 16; o > 0; o >>= 1) v = merge(v, shfl_down(v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // sh is reused across calls
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : Mom{0.0, 0.0, 0.0};
    for (int o = 16; o > 0; o >>= 1) v = merge(v, shfl_down(v, o));
  }
  return v;
}

// partial[b * (2D + 1) + e]: block b's mean_j (e = j), M2_j (e = D + j) and count (e = 2D)
template <class T>
__global__ void __launch_bounds__(kMomThreads)
    k_moments_partial(long long N, int D, int layout, int S, int slot, const T* out,
                      const signed char* status, double* partial) {
  __shared__ Mom sh[32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  double* mine = partial + (long long)blockIdx.x * (2 * D + 1);
  for (int j = 0; j < D; ++j) {
    double K = 0.0, s1 = 0.0, s2 = 0.0, c = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
      if (status && status[i] != 0) continue;
      const long long k = layout == ENS_LAYOUT_SOA ? ((long long)slot * D + j) * N + i
                                                   : (i * S + slot) * (long long)D + j;
      const double x = (double)out[k];
      if (c == 0.0) K = x;
      const double y = x - K;
      s1 += y;
      s2 = fma(y, y, s2);
      c += 1.0;
    }
    Mom v{0.0, 0.0, 0.0};
    if (c > 0.0) {
      const double d = s1 / c;  // mean - K
      v = Mom{c, K + d, fma(-s1, d, s2)};
    }
    v = block_merge(v, sh);
    if (threadIdx.x == 0) {
      mine[j] = v.mean;
      mine[D + j] = v.m2;
      if (j == 0) mine[2 * D] = v.n;
    }
  }
}

__global__ void __launch_bounds__(kMomThreads)
    k_moments_final(int D, int G, const double* partial, double* res) {
  __shared__ Mom sh[32];
  const int E = 2 * D + 1;
  for (int j = 0; j < D; ++j) {
    Mom v{0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
      const double* q = partial + (long long)b * E;
      v = merge(v, Mom{q[2 * D], q[j], q[D + j]});
    }
    v = block_merge(v, sh);
    if (threadIdx.x == 0) {
      res[j] = v.mean;
      res[D + j] = v.m2;
      if (j == 0) res[2 * D] = v.n;
    }
  }
}

}  // namespace
}  // namespace ens

using namespace ens;

extern "C" int ens_moments(long long N, int D, int dtype, int layout, int S, int slot,
                           const void* out, const signed char* status, double* scratch,
                           double* result, void* cuda_stream) {
  if (N < 0 || D < 1 || S < 1) return set_last_error(ENS_EINVAL, "bad sizes");
  if (slot < 0 || slot >= S) return set_last_error(ENS_EINVAL, "slot out of range");
  if (dtype != ENS_F32 && dtype != ENS_F64) return set_last_error(ENS_EINVAL, "unknown dtype");
  if (layout != ENS_LAYOUT_SOA && layout != ENS_LAYOUT_ROWMAJOR)
    return set_last_error(ENS_EINVAL, "unknown layout");
  if (!result || !scratch || (N > 0 && !out)) return set_last_error(ENS_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int G = ENS_MOMENTS_BLOCKS;
  if (dtype == ENS_F32)
    k_moments_partial<float><<<G, kMomThreads, 0, s>>>(
        N, D, layout, S, slot, static_cast<const float*>(out), status, scratch);
  else
    k_moments_partial<double><<<G, kMomThreads, 0, s>>>(
        N, D, layout, S, slot, static_cast<const double*>(out), status, scratch);
  k_moments_final<<<1, kMomThreads, 0, s>>>(D, G, scratch, result);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ENS_OK : set_last_error(ENS_ECUDA, cudaGetErrorString(e));
}

extern "C" int ens_moments_combine(int n_parts, int D, const double* parts, double* result) {
  if (n_parts < 1 || D < 1) return set_last_error(ENS_EINVAL, "bad sizes");
  if (!parts || !result) return set_last_error(ENS_EINVAL, "null pointer");
  const int E = 2 * D + 1;
  for (int j = 0; j < D; ++j) {  // the update of the kernels, over the parts in order
    double n = 0.0, mean = 0.0, m2 = 0.0;
    for (int r = 0; r < n_parts; ++r) {
      const double* q = parts + (long long)r * E;
      const double nb = q[2 * D], tot = n + nb;
      if (tot == 0.0) continue;
      const double d = q[j] - mean, fb = nb / tot;
      m2 = std::fma(d * d * n, fb, m2 + q[D + j]);
      mean = std::fma(d, fb, mean);
      n = tot;
    }
    result[j] = mean;
    result[D + j] = m2;
    if (j == 0) result[2 * D] = n;
  }
  return ENS_OK;
}
