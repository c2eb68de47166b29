// adjoint.cu -- instantiation and launch of the discrete-adjoint kernels (adjoint.cuh) for every
// (model, precision, method) pair.
#include "adjoint.cuh"

namespace ens {

namespace {

template <class RHS, class T, class TAB>
cudaError_t adj_launch(int which, const AdjArgs& a, cudaStream_t s) {
  // 64-thread blocks: a 65,536-trajectory ensemble becomes 1,024 blocks, ~6.7 per SM, so the
  // last wave is a small share of the work
  const int block = 64;
  const long long grid = (a.N + block - 1) / block;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (which == 0) k_adj_forward<RHS, T, TAB><<<(unsigned)grid, block, 0, s>>>(a);
  else k_adj_backward<RHS, T, TAB><<<(unsigned)grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <class T, class TAB>
cudaError_t adj_model(int which, int rhs_id, const AdjArgs& a, cudaStream_t s, bool* sup) {
  *sup = true;
  switch (rhs_id) {
    case ENS_RHS_LORENZ: return adj_launch<Lorenz<T>, T, TAB>(which, a, s);
    case ENS_RHS_ROBERTSON: return adj_launch<Robertson<T>, T, TAB>(which, a, s);
    case ENS_RHS_GBM: return adj_launch<GBM<T>, T, TAB>(which, a, s);
  }
  *sup = false;
  return cudaSuccess;
}

template <class T>
cudaError_t adj_alg(int which, int rhs_id, int alg, const AdjArgs& a, cudaStream_t s, bool* sup) {
  if (alg == ENS_TSIT5_FIXED) return adj_model<T, TabTsit5>(which, rhs_id, a, s, sup);
  if (alg == ENS_RK4) return adj_model<T, TabRK4>(which, rhs_id, a, s, sup);
  *sup = false;
  return cudaSuccess;
}

}  // namespace

int adjoint_stages(int alg) {
  return alg == ENS_TSIT5_FIXED ? TabTsit5::S : alg == ENS_RK4 ? TabRK4::S : 0;
}

cudaError_t launch_adjoint(int which, int rhs_id, int alg, int dtype, const AdjArgs& a,
                           cudaStream_t s, bool* sup) {
  if (dtype == ENS_F32) return adj_alg<float>(which, rhs_id, alg, a, s, sup);
  if (dtype == ENS_F64) return adj_alg<double>(which, rhs_id, alg, a, s, sup);
  *sup = false;
  return cudaSuccess;
}

}  // namespace ens
