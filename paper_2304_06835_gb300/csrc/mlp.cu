// mlp.cu -- the learned surrogate: a BF16 multilayer perceptron on the tcgen05 tensor cores.
//
// Not in the paper (an addition to the ensemble method): the network maps a Lorenz problem
// x = (sigma, rho, beta, u0) to the state u(tf) and is trained on solver output.  Widths
// 6 -> 256 -> 256 -> 256 -> 3, exact-erf GELU, BF16 operands with FP32 accumulation:
//   x_n = bf16(2 (x - lo)/(hi - lo) - 1),  Z_l = H_{l-1} W_l^T + b_l,  H_l = bf16(gelu(Z_l)),
//   y = Z_4 * y_std + y_mean.
// Training minimises the mean squared error on standardised targets with Adam; the backward
// pass is  dZ_4 = bf16(2 (Z_4 - t)/(3B)),  dW_l = dZ_l^T H_{l-1},  db_l = sum_b dZ_l,
// dZ_{l-1} = bf16((dZ_l W_l) * gelu'(Z_{l-1})).
//
// Every matrix product runs in one kernel, k_gemm: a CTA owns a 128-row tile of the output
// and BN columns; K is walked in 64-wide stages loaded by cp.async into the no-swizzle
// core-matrix layout (double-buffered), one thread issues tcgen05.mma (M = 128, N = BN,
// K = 16 per instruction) into an FP32 accumulator in tensor memory, and the epilogue reads it
// back with tcgen05.ld and applies bias / GELU / GELU' / affine output in registers.  The
// weight gradients contract over the batch with both operands MN-major (no transposed
// copies), split over K into deterministic partial sums.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda_bf16.h>

#include "ens_device.cuh"
#include "ens_internal.h"
#include "umma.cuh"

typedef __nv_bfloat16 bf16;

namespace ens {
namespace mlp {

constexpr int PAD_IN = 16, PAD_OUT = 16, HID = 256;
// flat FP32 parameter layout: W_1 [256][6], b_1, W_2 [256][256], b_2, W_3, b_3, W_4 [3][256], b_4
constexpr long long OFF_W1 = 0, OFF_B1 = OFF_W1 + 256 * 6;
constexpr long long OFF_W2 = OFF_B1 + 256, OFF_B2 = OFF_W2 + 256 * 256;
constexpr long long OFF_W3 = OFF_B2 + 256, OFF_B3 = OFF_W3 + 256 * 256;
constexpr long long OFF_W4 = OFF_B3 + 256, OFF_B4 = OFF_W4 + 3 * 256;
constexpr long long NP = OFF_B4 + 3;          // 134,147 parameters per member
// padded BF16 weights per member: W1b [256][16], W2b [256][256], W3b [256][256], W4b [16][256]
constexpr long long WB1 = 0, WB2 = WB1 + 256 * 16, WB3 = WB2 + 256 * 256, WB4 = WB3 + 256 * 256;
constexpr long long NWB = WB4 + 16 * 256;
// padded FP32 biases per member: b1 [256], b2 [256], b3 [256], b4 [16]
constexpr long long BB1 = 0, BB2 = 256, BB3 = 512, BB4 = 768, NBB = 784;

// ------------------------------------------------------------------------------ GEMM kernel
enum { EPI_AFFINE = 0, EPI_GELU_FWD = 1, EPI_GELU_BWD = 2, EPI_PARTIAL = 3 };

struct GemmArgs {
  int M, N, K;             // C[M][N] = sum_k A(m,k) B(n,k)
  const bf16* A;
  long long lda;
  int a_mn;                // 0: A(m,k) = A[m*lda + k]; 1: A(m,k) = A[k*lda + m]
  const bf16* B;
  long long ldb;
  int b_mn;                // 0: B(n,k) = B[n*ldb + k]; 1: B(n,k) = B[k*ldb + n]
  int epi;
  const float* bias;       // [N] or null
  const float* scale;      // EPI_AFFINE: [N] or null (1)
  const float* shift;      // EPI_AFFINE: [N] or null (0)
  const float* aux;        // EPI_GELU_BWD: Z [M][ldaux]
  long long ldaux;
  float* out_f32;          // EPI_AFFINE / EPI_PARTIAL / (EPI_GELU_FWD: Z, optional)
  long long ldo;
  long long split_stride;  // EPI_PARTIAL: elements between the partial sums of splits
  bf16* out_bf16;          // EPI_GELU_FWD: H; EPI_GELU_BWD: dZ
  long long ldob;
  int k_chunk;             // split-K: CTA z covers K range [z*k_chunk, (z+1)*k_chunk)
  int* err;                // set to 1 when a wait for the tensor cores times out
};

constexpr int BM = 128, BK = 64, NTHREADS = 256;

// erf for the GELU by Abramowitz & Stegun 7.1.26 (Hastings' rational approximation):
//   erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2},  t = 1 / (1 + p x),  x >= 0,
// |error| <= 1.5e-7, four orders below the bf16 resolution (2^-9) of the stored activations.
// Branch-free (CUDA's erff branches on |x| and diverges inside warps); e^{-x^2} is returned
// too, since gelu' needs phi(z) = e^{-z^2/2} / sqrt(2 pi) with the same exponential.
__device__ __forceinline__ float erf_as(float x, float* ex) {
  const float ax = fabsf(x);
  const float t = __fdividef(1.f, fmaf(0.3275911f, ax, 1.f));
  float q = fmaf(1.061405429f, t, -1.453152027f);
  q = fmaf(q, t, 1.421413741f);
  q = fmaf(q, t, -0.284496736f);
  q = fmaf(q, t, 0.254829592f);
  q *= t;
  const float e = ex2_approx(-(ax * ax) * 1.4426950408889634f);  // e^{-x^2}
  *ex = e;
  return copysignf(fmaf(-q, e, 1.f), x);
}
// gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2   (Hendrycks & Gimpel, exact erf form)
__device__ __forceinline__ float gelu_f(float z) {
  float e;
  const float er = erf_as(z * 0.70710678118654752440f, &e);
  return 0.5f * z * (1.f + er);
}
// gelu'(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad_f(float z) {
  float e;
  const float er = erf_as(z * 0.70710678118654752440f, &e);
  return fmaf(z * 0.39894228040143267794f, e, 0.5f * (1.f + er));
}

// The same two functions on a pair of values with the paired FP32 instructions (FFMA2 / FMUL2 /
// FADD2 round each half exactly like the scalar instruction, so each lane equals gelu_f /
// gelu_grad_f of that value); the approximate reciprocal and exponential stay per lane.
__device__ __forceinline__ float2 erf_as2(float2 x, float2* ex) {
  const float2 ax = make_float2(fabsf(x.x), fabsf(x.y));
  const float2 den = __ffma2_rn(make_float2(0.3275911f, 0.3275911f), ax, make_float2(1.f, 1.f));
  const float2 t = make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y));
  float2 q = __ffma2_rn(make_float2(1.061405429f, 1.061405429f), t,
                        make_float2(-1.453152027f, -1.453152027f));
  q = __ffma2_rn(q, t, make_float2(1.421413741f, 1.421413741f));
  q = __ffma2_rn(q, t, make_float2(-0.284496736f, -0.284496736f));
  q = __ffma2_rn(q, t, make_float2(0.254829592f, 0.254829592f));
  q = __fmul2_rn(q, t);
  const float2 a2 = __fmul2_rn(__fmul2_rn(ax, ax), make_float2(-1.4426950408889634f,
                                                                -1.4426950408889634f));
  const float2 e = make_float2(ex2_approx(a2.x), ex2_approx(a2.y));
  *ex = e;
  const float2 y = __ffma2_rn(make_float2(-q.x, -q.y), e, make_float2(1.f, 1.f));
  return make_float2(copysignf(y.x, x.x), copysignf(y.y, x.y));
}
__device__ __forceinline__ float2 gelu_f2(float2 z) {
  float2 e;
  const float2 er = erf_as2(__fmul2_rn(z, make_float2(0.70710678118654752440f,
                                                      0.70710678118654752440f)), &e);
  return __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), z), __fadd2_rn(make_float2(1.f, 1.f), er));
}
__device__ __forceinline__ float2 gelu_grad_f2(float2 z) {
  float2 e;
  const float2 er = erf_as2(__fmul2_rn(z, make_float2(0.70710678118654752440f,
                                                      0.70710678118654752440f)), &e);
  return __ffma2_rn(__fmul2_rn(z, make_float2(0.39894228040143267794f, 0.39894228040143267794f)),
                    e, __fmul2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(make_float2(1.f, 1.f), er)));
}

// (test aid) out[i] = gelu(z[i]) (which = 0) or gelu'(z[i]) (which = 1) as the kernels compute
__global__ void k_activation(int which, long long n, const float* __restrict__ z,
                             float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = which ? gelu_grad_f(z[i]) : gelu_f(z[i]);
}

template <int BN>
struct Tile {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = 2 * STAGE + 1024;  // + alignment slack
  static constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
  // K-major: core matrices along K adjacent (128 B), 8-row groups BK/8 * 128 = 1024 B apart
  static constexpr uint32_t KM_LBO = 128, KM_SBO = (BK / 8) * 128;
  // MN-major: core matrices along MN adjacent (128 B), 8-k groups (rows/8)*128 B apart
  static constexpr uint32_t A_MN_LBO = (BM / 8) * 128, B_MN_LBO = (BN / 8) * 128, MN_SBO = 128;
};

// One 64-wide K stage of both operands, 16-byte cp.async pieces.  Thread order inside a
// warp: the 8 rows of a core matrix fastest, then 4 neighbouring core matrices, so a warp
// fills 512 contiguous bytes of shared memory (no bank conflicts) while reading 64
// contiguous bytes (two full sectors) from each of 8 global rows.
template <int ROWS>
__device__ __forceinline__ void load_kmajor(uint32_t dst, const bf16* src, long long ld, int r0,
                                            int rlim, int k0, int kend, uint32_t sbo) {
  // K-major tile [ROWS][BK]: piece (row, kc) -> (row/8)*sbo + kc*128 + (row%8)*16.  Thread t
  // owns kc = (t/8)%8 and rows (t/64)*8 + t%8 + 32 i, i < ROWS/32 (constant trip count).
  constexpr int PIECES = ROWS * (BK / 8);
  constexpr int IT = (PIECES + NTHREADS - 1) / NTHREADS;
  const int t = threadIdx.x, lo = t & 7, kc = (t >> 3) & 7, row0 = (t >> 6) * 8 + lo;
  if (PIECES < NTHREADS && t >= PIECES) return;  // small tile: the first PIECES threads
  const int gk = k0 + kc * 8;
  const bool kok = gk < kend;
  const bf16* p = src + (long long)(r0 + row0) * ld + gk;
  const long long step = 32 * ld;
  uint32_t d = dst + (t >> 6) * sbo + kc * 128 + lo * 16;
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const bool ok = kok && (r0 + row0 + 32 * i) < rlim;
    umma::cp_async16(d, ok ? p : src, ok ? 16 : 0);
    p += step;
    d += 4 * sbo;
  }
}
template <int ROWS>
__device__ __forceinline__ void load_mnmajor(uint32_t dst, const bf16* src, long long ld, int r0,
                                             int rlim, int k0, int kend, uint32_t lbo) {
  // MN-major tile (ROWS along M/N, BK along K): piece (k, rc) -> (k/8)*lbo + rc*128 +
  // (k%8)*16.  Thread t owns k%8 = t%8; pieces walk rc fastest, then the k groups.
  constexpr int RC = ROWS / 8;
  constexpr int PIECES = BK * RC;
  constexpr int IT = (PIECES + NTHREADS - 1) / NTHREADS;
  const int t = threadIdx.x, lo = t & 7;
  if (PIECES < NTHREADS && t >= PIECES) return;  // small tile: the first PIECES threads
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int rest = (t >> 3) + i * (NTHREADS / 8);
    const int rc = rest % RC, hi = rest / RC;
    const int gk = k0 + hi * 8 + lo, gr = r0 + rc * 8;
    const bool ok = gk < kend && gr < rlim;
    umma::cp_async16(dst + hi * lbo + rc * 128 + lo * 16,
                     ok ? src + (long long)gk * ld + gr : src, ok ? 16 : 0);
  }
}

template <int BN>
__device__ __forceinline__ void load_stage(const GemmArgs& g, unsigned char* sA, unsigned char* sB,
                                           int m0, int n0, int k0, int kend) {
  typedef Tile<BN> TL;
  const uint32_t a = umma::smem_addr(sA), b = umma::smem_addr(sB);
  if (!g.a_mn) load_kmajor<BM>(a, g.A, g.lda, m0, g.M, k0, kend, TL::KM_SBO);
  else load_mnmajor<BM>(a, g.A, g.lda, m0, g.M, k0, kend, TL::A_MN_LBO);
  if (!g.b_mn) load_kmajor<BN>(b, g.B, g.ldb, n0, g.N, k0, kend, TL::KM_SBO);
  else load_mnmajor<BN>(b, g.B, g.ldb, n0, g.N, k0, kend, TL::B_MN_LBO);
}

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 2) k_gemm(const GemmArgs g) {
  typedef Tile<BN> TL;
  extern __shared__ unsigned char smraw[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tslot;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * g.k_chunk;
  const int kend = min(g.K, kbeg + g.k_chunk);
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;

  if (tid == 0) {
    umma::mbar_init(&bar[0], 1);
    umma::mbar_init(&bar[1], 1);
    umma::mbar_init_fence();
  }
  if (warp == 0) umma::tmem_alloc<TL::TCOLS>(&tslot);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tacc = tslot;
  const uint32_t idesc = umma::idesc_bf16(BM, BN, g.a_mn, g.b_mn);

  bool ok = true;
  if (nk > 0) {
    load_stage<BN>(g, sm, sm + TL::A_BYTES, m0, n0, kbeg, kend);
    umma::cp_async_commit();
  }
  // Waits for the tensor cores are done by one thread; __syncthreads_and releases the block
  // and shares the outcome (polling by every thread would take issue slots from the other
  // resident block's epilogue).
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int s = kt & 1;
    if (kt + 1 < nk) {
      if (kt >= 1) {
        bool w = true;
        if (tid == 0) w = umma::mbar_wait(&bar[s ^ 1], ((kt - 1) >> 1) & 1);
        ok = __syncthreads_and(w);
      }
      if (!ok) break;
      unsigned char* st = sm + (s ^ 1) * TL::STAGE;
      load_stage<BN>(g, st, st + TL::A_BYTES, m0, n0, kbeg + (kt + 1) * BK, kend);
      umma::cp_async_commit();
      umma::cp_async_wait<1>();
    } else {
      umma::cp_async_wait<0>();
    }
    umma::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      umma::fence_after();
      const uint32_t a = umma::smem_addr(sm + s * TL::STAGE);
      const uint32_t b = a + TL::A_BYTES;
      const int k0 = kbeg + kt * BK;
      const int steps = min(BK / 16, (kend - k0 + 15) / 16);
      for (int j = 0; j < steps; ++j) {
        const uint64_t ad = g.a_mn ? umma::desc(a + j * 2 * TL::A_MN_LBO, TL::A_MN_LBO, TL::MN_SBO)
                                   : umma::desc(a + j * 256, TL::KM_LBO, TL::KM_SBO);
        const uint64_t bd = g.b_mn ? umma::desc(b + j * 2 * TL::B_MN_LBO, TL::B_MN_LBO, TL::MN_SBO)
                                   : umma::desc(b + j * 256, TL::KM_LBO, TL::KM_SBO);
        umma::mma_bf16(tacc, ad, bd, idesc, (kt > 0 || j > 0) ? 1u : 0u);
      }
      umma::mma_commit(&bar[s]);
    }
  }
  if (nk > 0 && ok) {
    bool w = true;
    if (tid == 0) w = umma::mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1);
    ok = __syncthreads_and(w);
  }
  if (!ok) {
    if (tid == 0) atomicExch(g.err, 1);
    umma::cp_async_wait<0>();
    // give any MMA still in flight a bounded chance to finish before the memory goes away
    if (nk > 0) umma::mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1, 100000000ull);
  }
  umma::fence_after();

  // Epilogue, in passes of QW columns staged through the (now idle) operand shared memory:
  // warps w and w + 4 read TMEM lane quarter w & 3 (rows 32 (w & 3) + lane of the tile),
  // alternating 16-column chunks; the staged pass is then written to global memory by all
  // threads in row-contiguous (coalesced) pieces.
  constexpr int QW = BN < 64 ? BN : 64;
  constexpr int ZS = QW + 4, HS = QW + 8;  // staging row strides (floats, bf16)
  float* zst = reinterpret_cast<float*>(sm);
  bf16* hst = reinterpret_cast<bf16*>(sm + BM * ZS * 4);
  const int lq = warp & 3, half = warp >> 2;
  const int r = lq * 32 + lane;
  const bool fp32_out = g.out_f32 != nullptr && g.epi != EPI_GELU_BWD;
  const bool bf16_out = g.epi == EPI_GELU_FWD || g.epi == EPI_GELU_BWD;
  float* obase = g.out_f32 ? g.out_f32 + (g.epi == EPI_PARTIAL
                                              ? (long long)blockIdx.z * g.split_stride : 0LL)
                           : nullptr;
  for (int q = 0; q < BN / QW; ++q) {
    const int cb = q * QW;  // first column of the pass within the tile
    if (g.epi == EPI_GELU_BWD) {  // stage the pre-activations Z of this pass (coalesced)
      for (int i = tid; i < BM * QW; i += NTHREADS) {
        const int rr = i / QW, cc = i % QW, gr = m0 + rr, gc = n0 + cb + cc;
        zst[rr * ZS + cc] =
            (gr < g.M && gc < g.N) ? __ldg(g.aux + (long long)gr * g.ldaux + gc) : 0.f;
      }
      __syncthreads();
    }
    for (int c16 = (QW >= 32 ? half : 0); c16 < QW / 16; c16 += (QW >= 32 ? 2 : QW / 16)) {
      if (QW < 32 && half) break;  // a 16-wide tile needs one warp per lane quarter
      uint32_t rv[16];
      if (nk > 0) {
        umma::tmem_ld16(tacc + ((uint32_t)(lq * 32) << 16) + cb + c16 * 16, rv);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) rv[j] = 0u;
      }
      const int c0 = c16 * 16, nb = n0 + cb + c0;
      const bool full = nb + 16 <= g.N;  // no column of this chunk is past N
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = ok ? __uint_as_float(rv[j]) : 0.f;
      if (g.bias && g.epi != EPI_PARTIAL) {
        if (full) {  // 16 biases as four 16-byte loads (the bias arrays are 16-byte aligned)
          const float4* b4 = reinterpret_cast<const float4*>(g.bias + nb);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 b = __ldg(b4 + j);
            const float2 s0 = __fadd2_rn(make_float2(v[4 * j], v[4 * j + 1]), make_float2(b.x, b.y));
            const float2 s1 =
                __fadd2_rn(make_float2(v[4 * j + 2], v[4 * j + 3]), make_float2(b.z, b.w));
            v[4 * j] = s0.x;
            v[4 * j + 1] = s0.y;
            v[4 * j + 2] = s1.x;
            v[4 * j + 3] = s1.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (nb + j < g.N) v[j] += __ldg(g.bias + nb + j);
        }
      }
      if (g.epi == EPI_AFFINE) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (nb + j < g.N) {
            const float sc = g.scale ? __ldg(g.scale + nb + j) : 1.f;
            const float sh = g.shift ? __ldg(g.shift + nb + j) : 0.f;
            v[j] = fmaf(v[j], sc, sh);
          }
      }
      if (fp32_out) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(zst + r * ZS + c0 + j) =
              make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
      if (bf16_out) {
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          float2 ab;
          if (g.epi == EPI_GELU_FWD) {
            ab = gelu_f2(make_float2(v[j], v[j + 1]));
          } else {
            const float2 z2 = *reinterpret_cast<const float2*>(zst + r * ZS + c0 + j);
            ab = __fmul2_rn(make_float2(v[j], v[j + 1]), gelu_grad_f2(z2));
          }
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(ab.x, ab.y);
          pk[j / 2] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(hst + r * HS + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4*>(hst + r * HS + c0 + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
    }
    __syncthreads();
    // write the pass: rows m0 .. m0 + 127, columns n0 + cb .. n0 + cb + QW - 1 (bounded)
    const int ncol = min(QW, g.N - (n0 + cb));
    if (ok && ncol > 0) {
      if (fp32_out) {
        const bool vec = (g.ldo % 4 == 0) && (((uintptr_t)obase & 15) == 0) && (ncol % 4 == 0) &&
                         ((n0 + cb) % 4 == 0);
        if (vec && ncol == QW) {  // full pass: constant width
          constexpr int VW = QW / 4;
#pragma unroll
          for (int i = tid; i < BM * VW; i += NTHREADS) {
            const int rr = i / VW, cc = (i % VW) * 4, gr = m0 + rr;
            if (gr < g.M)
              *reinterpret_cast<float4*>(obase + (long long)gr * g.ldo + n0 + cb + cc) =
                  *reinterpret_cast<const float4*>(zst + rr * ZS + cc);
          }
        } else if (vec) {
          const int vw = ncol / 4;
          for (int i = tid; i < BM * vw; i += NTHREADS) {
            const int rr = i / vw, cc = (i % vw) * 4, gr = m0 + rr;
            if (gr < g.M)
              *reinterpret_cast<float4*>(obase + (long long)gr * g.ldo + n0 + cb + cc) =
                  *reinterpret_cast<const float4*>(zst + rr * ZS + cc);
          }
        } else {
          for (int i = tid; i < BM * ncol; i += NTHREADS) {
            const int rr = i / ncol, cc = i % ncol, gr = m0 + rr;
            if (gr < g.M) obase[(long long)gr * g.ldo + n0 + cb + cc] = zst[rr * ZS + cc];
          }
        }
      }
      if (bf16_out) {
        const bool vec = (g.ldob % 8 == 0) && (((uintptr_t)g.out_bf16 & 15) == 0) &&
                         (ncol % 8 == 0) && ((n0 + cb) % 8 == 0);
        if (vec && ncol == QW) {  // full pass: constant width
          constexpr int VW = QW / 8;
#pragma unroll
          for (int i = tid; i < BM * VW; i += NTHREADS) {
            const int rr = i / VW, cc = (i % VW) * 8, gr = m0 + rr;
            if (gr < g.M)
              *reinterpret_cast<uint4*>(g.out_bf16 + (long long)gr * g.ldob + n0 + cb + cc) =
                  *reinterpret_cast<const uint4*>(hst + rr * HS + cc);
          }
        } else if (vec) {
          const int vw = ncol / 8;
          for (int i = tid; i < BM * vw; i += NTHREADS) {
            const int rr = i / vw, cc = (i % vw) * 8, gr = m0 + rr;
            if (gr < g.M)
              *reinterpret_cast<uint4*>(g.out_bf16 + (long long)gr * g.ldob + n0 + cb + cc) =
                  *reinterpret_cast<const uint4*>(hst + rr * HS + cc);
          }
        } else {
          for (int i = tid; i < BM * ncol; i += NTHREADS) {
            const int rr = i / ncol, cc = i % ncol, gr = m0 + rr;
            if (gr < g.M) g.out_bf16[(long long)gr * g.ldob + n0 + cb + cc] = hst[rr * HS + cc];
          }
        }
      }
    }
    __syncthreads();
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) {
    umma::fence_after();
    umma::tmem_dealloc<TL::TCOLS>(tacc);
  }
}

// ------------------------------------------------------------------------------ small kernels
struct Box {
  float lo[6], inv[6];  // inv = 2 / (hi - lo)
  float hi[6];
};

// x_n = bf16(2 (x - lo)/(hi - lo) - 1), columns 6..15 zero; row b reads x[idx[b]] when an
// index array is given (minibatch gather)
__global__ void k_input(long long B, const float* __restrict__ x, const long long* __restrict__ idx,
                        Box box, bf16* __restrict__ xn) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * PAD_IN) return;
  const long long b = i / PAD_IN;
  const long long r = idx ? idx[b] : b;
  const int c = (int)(i % PAD_IN);
  float v = 0.f;
  if (c < 6) v = (x[r * 6 + c] - box.lo[c]) * box.inv[c] - 1.f;
  xn[i] = __float2bfloat16_rn(v);
}

// loss partial sums and dZ_4 = bf16(2 (z - t) / (3 B)); t = (y - mean)/std
__global__ void k_loss(long long B, const float* __restrict__ z4, const float* __restrict__ y,
                       const long long* __restrict__ idx, const float* __restrict__ mean,
                       const float* __restrict__ stdv, bf16* __restrict__ dz4, double* loss) {
  __shared__ double red[256];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < B * PAD_OUT) {
    const long long b = i / PAD_OUT;
    const int c = (int)(i % PAD_OUT);
    float d = 0.f;
    if (c < 3) {
      const long long row = idx ? idx[b] : b;
      const float t = (y[row * 3 + c] - mean[c]) / stdv[c];
      const float r = z4[b * PAD_OUT + c] - t;
      acc = (double)r * r;
      d = 2.f * r / (3.f * (float)B);
    }
    dz4[i] = __float2bfloat16_rn(d);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0] / (3.0 * (double)B));
}

// column sums of a bf16 matrix [rows][ld] over a chunk of rows: part[chunk][c]
__global__ void k_colsum(long long rows, int ncols, long long ld, const bf16* __restrict__ a,
                         long long chunk, float* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const long long r0 = (long long)blockIdx.y * chunk;
  const long long r1 = min(rows, r0 + chunk);
  float s = 0.f;
  for (long long r = r0; r < r1; ++r) s += __bfloat162float(a[r * ld + c]);
  part[(long long)blockIdx.y * ncols + c] = s;
}

// out[r * out_ld + c] = sum_s part[s * stride + r * ld + c]   (r < rows, c < cols)
__global__ void k_reduce(int S, long long stride, int rows, int cols, long long ld,
                         const float* __restrict__ part, float* __restrict__ out, long long out_ld) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  float s = 0.f;
  for (int k = 0; k < S; ++k) s += part[k * stride + (long long)r * ld + c];
  out[(long long)r * out_ld + c] = s;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 padded weights and padded FP32 biases of one member from its FP32 parameters
__global__ void k_refresh(const float* __restrict__ p, bf16* __restrict__ wb, float* __restrict__ bb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NWB) {
    float v = 0.f;
    if (i < WB2) {
      const long long r = i / 16, c = i % 16;
      v = c < 6 ? p[OFF_W1 + r * 6 + c] : 0.f;
    } else if (i < WB3) {
      v = p[OFF_W2 + (i - WB2)];
    } else if (i < WB4) {
      v = p[OFF_W3 + (i - WB3)];
    } else {
      const long long r = (i - WB4) / 256, c = (i - WB4) % 256;
      v = r < 3 ? p[OFF_W4 + r * 256 + c] : 0.f;
    }
    wb[i] = __float2bfloat16_rn(v);
  }
  if (i < NBB) {
    float v;
    if (i < BB2) v = p[OFF_B1 + i];
    else if (i < BB3) v = p[OFF_B2 + (i - BB2)];
    else if (i < BB4) v = p[OFF_B3 + (i - BB3)];
    else v = (i - BB4) < 3 ? p[OFF_B4 + (i - BB4)] : 0.f;
    bb[i] = v;
  }
}

// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for every weight and bias, from Philox4x32-10
// (counter = (parameter index, member, 0x4D4C5000), key = seed).
__global__ void k_init(long long n, int member, unsigned long long seed, float* __restrict__ p) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 x = Philox::gen(make_uint4((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)member,
                                         0x4D4C5000u),
                              make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float u = ((float)(x.x >> 8) + 0.5f) * 5.9604644775390625e-08f;  // (0, 1)
  const int fan_in = i < OFF_W2 ? 6 : 256;
  p[i] = (2.f * u - 1.f) * rsqrtf((float)fan_in);
}

// mean and population standard deviation over the members; fallback when the input leaves
// the training box or max_j std_j > tau.  A fallback sample is appended (slot from an atomic
// counter) to the compacted solver problem: index, params (sigma, rho, beta), u0, tspan.
struct Compact {
  long long* index;   // [B] or null (no compaction)
  float* params;      // [B][3]
  float* u0;          // [B][3]
  float* tspan;       // [B][2]
  float t0, t1;
};

__global__ void k_gate(long long B, int E, const float* __restrict__ x,
                       const float* __restrict__ ym, Box box, float tau, float* __restrict__ mean,
                       float* __restrict__ spread, unsigned char* __restrict__ fb, unsigned long long* n_fb, Compact cp) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool f = false;
  if (b < B) {
    bool out = false;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float v = x[b * 6 + c];
      out = out || !(v >= box.lo[c] && v <= box.hi[c]);
    }
    float smax = 0.f;
    for (int j = 0; j < 3; ++j) {
      float s = 0.f;
      for (int e = 0; e < E; ++e) s += ym[((long long)e * B + b) * 3 + j];
      const float mu = s / (float)E;
      float q = 0.f;
      for (int e = 0; e < E; ++e) {
        const float d = ym[((long long)e * B + b) * 3 + j] - mu;
        q += d * d;
      }
      smax = fmaxf(smax, sqrtf(q / (float)E));
      if (mean) mean[b * 3 + j] = mu;
    }
    if (spread) spread[b] = smax;
    f = out || !(smax <= tau);
    fb[b] = f ? 1 : 0;
  }
  // warp-aggregated slot reservation for the compacted problem
  const unsigned ballot = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0 && ballot && n_fb) base = atomicAdd(n_fb, (unsigned long long)__popc(ballot));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (f && cp.index && n_fb) {
    const unsigned long long pos = base + __popc(ballot & ((1u << lane) - 1u));
    cp.index[pos] = b;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cp.params[pos * 3 + c] = x[b * 6 + c];
      cp.u0[pos * 3 + c] = x[b * 6 + 3 + c];
    }
    cp.tspan[pos * 2] = cp.t0;
    cp.tspan[pos * 2 + 1] = cp.t1;
  }
}

// y[index[i]] = u[i] for the n solved fallback samples (row-major [n][3])
__global__ void k_scatter(long long n, const long long* __restrict__ index,
                          const float* __restrict__ u, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 3) return;
  y[index[i / 3] * 3 + i % 3] = u[i];
}


// ------------------------------------------------------------------------------ fused forward
// Inference of all members in one persistent kernel with the activations kept on chip.  A CTA
// owns two 128-sample tiles at a time (slots 0 and 1), each with its own FP32 accumulator in
// TMEM (256 columns) and its own activation buffer H in shared memory (128 x 256 bf16 in the
// K-major core-matrix layout the next layer's MMA reads).  Warp roles:
//   warp 0      producer: TMA bulk copies of the input tiles and of the weight chunks (packed
//               beforehand in the exact shared-memory layout) into S stage buffers;
//   warp 1      MMA issuer: per (member, layer, slot) the K-chunks of tcgen05.mma, committing
//               each stage back to the producer and the finished accumulator to the epilogue;
//   warps 2-17  four epilogue groups of four warps, two per slot (alternate 16-column
//               chunks; a group's warps cover the four TMEM lane quarters): TMEM -> bias,
//               GELU -> bf16 H (or, after the last layer, y = (z + b4) * y_std + y_mean).
// Jobs run in the order member, layer, slot, so the MMAs of one slot overlap the epilogue of
// the other.  The arithmetic per output equals the layer-by-layer k_gemm path (same K order,
// same epilogue operations), so the results are identical.
namespace fused {
constexpr int S = 2;                                  // weight stages
constexpr int NT = 576;                               // 18 warps: producer, MMA, 16 epilogue
constexpr uint32_t H_BYTES = 65536, X_BYTES = 4096, W_BYTES = 32768;
constexpr uint32_t OFF_X = 2 * H_BYTES, OFF_W = OFF_X + 2 * X_BYTES;
constexpr uint32_t SMEM = OFF_W + S * W_BYTES + 1024;  // dynamic shared memory (+ alignment)
constexpr long long NWP = 139264;                     // packed bf16 weights per member
// layer l streams nchunks(l) chunks: W1 whole (8 KB), W2 / W3 in K-chunks of 64 (32 KB),
// W4 whole (8 KB)
__host__ __device__ constexpr int nchunks(int l) { return (l == 1 || l == 2) ? 4 : 1; }
__host__ __device__ constexpr uint32_t chunk_bytes(int l) {
  return (l == 1 || l == 2) ? 32768u : 8192u;
}
__host__ __device__ constexpr long long woff(int l) {  // bf16 elements
  return l == 0 ? 0 : l == 1 ? 4096 : l == 2 ? 69632 : 135168;
}
}  // namespace fused

// element offset of (n, k) in a K-major core-matrix tile whose 8-row groups are `sbo_el`
// elements apart
__device__ __forceinline__ long long cm_off(int n, int k, int sbo_el) {
  return (long long)(n >> 3) * sbo_el + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);
}

// Pack one member's weights for the fused kernel: W1 [256][16] (SBO 256 B), W2 and W3 as four
// K-chunks of [256][64] (SBO 1024 B), W4 [16][256] (SBO 4096 B), zero padding.
__global__ void k_pack(const float* __restrict__ p, bf16* __restrict__ wp) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fused::NWP) return;
  float v = 0.f;
  long long dst;
  if (i < 4096) {  // W1: n < 256, k < 16
    const int n = (int)(i / 16), k = (int)(i % 16);
    v = k < 6 ? p[OFF_W1 + n * 6 + k] : 0.f;
    dst = cm_off(n, k, 128);
  } else if (i < 4096 + 2 * 65536) {  // W2 / W3: n < 256, k < 256
    const long long j = (i - 4096) % 65536;
    const int which = (int)((i - 4096) / 65536);
    const int n = (int)(j / 256), k = (int)(j % 256);
    v = p[(which ? OFF_W3 : OFF_W2) + (long long)n * 256 + k];
    dst = fused::woff(1 + which) + (k / 64) * 16384 + cm_off(n, k % 64, 512);
  } else {  // W4: n < 16 (3 real), k < 256
    const long long j = i - 135168;
    const int n = (int)(j / 256), k = (int)(j % 256);
    v = n < 3 ? p[OFF_W4 + n * 256 + k] : 0.f;
    dst = fused::woff(3) + cm_off(n, k, 2048);
  }
  wp[dst] = __float2bfloat16_rn(v);
}

// Normalised inputs in tiles of 128 rows, each tile in the K-major core-matrix layout
// (SBO 256 B); rows past B are zero.
__global__ void k_input_tiled(long long B, long long rows, const float* __restrict__ x, Box box,
                              bf16* __restrict__ xt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * PAD_IN) return;
  const long long b = i / PAD_IN;
  const int c = (int)(i % PAD_IN);
  float v = 0.f;
  if (b < B && c < 6) v = (x[b * 6 + c] - box.lo[c]) * box.inv[c] - 1.f;
  xt[(b / 128) * 2048 + cm_off((int)(b % 128), c, 128)] = __float2bfloat16_rn(v);
}

struct FusedArgs {
  long long B;          // rows of this call (tiles cover ceil(B / 128) * 128 rows)
  long long ystride;    // rows of each member's block of y
  int ntiles, E;
  const bf16* xt;       // [ntiles][2048] tiled normalised inputs
  const bf16* wp;       // [E][NWP] packed weights
  const float* bias;    // [E][NBB] padded biases
  const float* ystat;   // y_mean[3], y_std[3]
  float* y;             // [E][B][3]
  int* err;
};

__global__ void __launch_bounds__(fused::NT, 1) k_mlp_fused(const FusedArgs f) {
  using namespace fused;
  extern __shared__ unsigned char smraw[];
  __shared__ uint64_t wfull[S], wempty[S], xfull[2], xempty[2], dfull[2], hready[2];
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = umma::smem_addr(sm);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npairs = (f.ntiles + 1) / 2;
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      umma::mbar_init(&wfull[i], 1);
      umma::mbar_init(&wempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&xfull[i], 1);
      umma::mbar_init(&xempty[i], 1);
      umma::mbar_init(&dfull[i], 1);
      umma::mbar_init(&hready[i], 256);
    }
    abort_flag = 0;
    umma::mbar_init_fence();
  }
  if (warp == 0) umma::tmem_alloc<512>(&tslot);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tbase = tslot;
  auto fail = [&]() {
    abort_flag = 1;
    atomicExch(f.err, 1);
  };

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- producer
    int use = 0, xuse[2] = {0, 0};
    for (int pr = blockIdx.x; pr < npairs && !abort_flag; pr += gridDim.x) {
      const int ns = (2 * pr + 1 < f.ntiles) ? 2 : 1;
      for (int sl = 0; sl < ns && !abort_flag; ++sl) {
        if (!umma::mbar_wait(&xempty[sl], (xuse[sl] & 1) ^ 1)) { fail(); break; }
        umma::mbar_arrive_expect_tx(&xfull[sl], X_BYTES);
        umma::bulk_g2s(sbase + OFF_X + sl * X_BYTES, f.xt + (long long)(2 * pr + sl) * 2048,
                       X_BYTES, &xfull[sl]);
        ++xuse[sl];
      }
      for (int m = 0; m < f.E && !abort_flag; ++m)
        for (int l = 0; l < 4 && !abort_flag; ++l)
          for (int sl = 0; sl < ns && !abort_flag; ++sl)
            for (int c = 0; c < nchunks(l); ++c) {
              const int st = use % S, n = use / S;
              if (!umma::mbar_wait(&wempty[st], (n & 1) ^ 1)) { fail(); break; }
              umma::mbar_arrive_expect_tx(&wfull[st], chunk_bytes(l));
              umma::bulk_g2s(sbase + OFF_W + st * W_BYTES,
                             f.wp + (long long)m * NWP + woff(l) + c * (chunk_bytes(l) / 2),
                             chunk_bytes(l), &wfull[st]);
              ++use;
            }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    int use = 0, J[2] = {0, 0}, xuse[2] = {0, 0};
    for (int pr = blockIdx.x; pr < npairs && !abort_flag; pr += gridDim.x) {
      const int ns = (2 * pr + 1 < f.ntiles) ? 2 : 1;
      for (int m = 0; m < f.E && !abort_flag; ++m)
        for (int l = 0; l < 4 && !abort_flag; ++l)
          for (int sl = 0; sl < ns && !abort_flag; ++sl) {
            if (J[sl] > 0 && !umma::mbar_wait(&hready[sl], (J[sl] - 1) & 1)) { fail(); break; }
            if (l == 0 && m == 0 && !umma::mbar_wait(&xfull[sl], xuse[sl] & 1)) { fail(); break; }
            umma::fence_after();
            const uint32_t tacc = tbase + sl * 256;
            const uint32_t hA = sbase + sl * H_BYTES;
            const uint32_t idesc = umma::idesc_bf16(128, l == 3 ? 16 : 256, 0, 0);
            for (int c = 0; c < nchunks(l) && !abort_flag; ++c) {
              const int st = use % S, n = use / S;
              if (!umma::mbar_wait(&wfull[st], n & 1)) { fail(); break; }
              umma::fence_after();
              const uint32_t wB = sbase + OFF_W + st * W_BYTES;
              if (l == 0) {
                umma::mma_bf16(tacc, umma::desc(sbase + OFF_X + sl * X_BYTES, 128, 256),
                               umma::desc(wB, 128, 256), idesc, 0u);
              } else if (l < 3) {
                for (int j = 0; j < 4; ++j)
                  umma::mma_bf16(tacc, umma::desc(hA + (c * 4 + j) * 256, 128, 4096),
                                 umma::desc(wB + j * 256, 128, 1024), idesc,
                                 (c > 0 || j > 0) ? 1u : 0u);
              } else {
                for (int j = 0; j < 16; ++j)
                  umma::mma_bf16(tacc, umma::desc(hA + j * 256, 128, 4096),
                                 umma::desc(wB + j * 256, 128, 4096), idesc, j > 0 ? 1u : 0u);
              }
              umma::mma_commit(&wempty[st]);
              ++use;
            }
            umma::mma_commit(&dfull[sl]);
            if (l == 0 && m == f.E - 1) {
              umma::mma_commit(&xempty[sl]);
              ++xuse[sl];
            }
            ++J[sl];
          }
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue groups
    const int grp = (warp - 2) >> 2, sl = grp >> 1, half = grp & 1, lq = warp & 3;
    const int r = lq * 32 + lane;
    int J = 0;
    for (int pr = blockIdx.x; pr < npairs && !abort_flag; pr += gridDim.x) {
      if (sl == 1 && 2 * pr + 1 >= f.ntiles) continue;
      const long long grow = (long long)(2 * pr + sl) * 128 + r;
      for (int m = 0; m < f.E && !abort_flag; ++m)
        for (int l = 0; l < 4 && !abort_flag; ++l) {
          // every lane waits; the outcome is made warp-uniform so that a time-out never
          // leaves part of a warp inside the warp-collective tcgen05.ld below
          const bool got = __all_sync(0xffffffffu, umma::mbar_wait(&dfull[sl], J & 1));
          if (!got) { fail(); break; }
          umma::fence_after();
          const uint32_t trow = tbase + sl * 256 + ((uint32_t)(lq * 32) << 16);
          const float* bias = f.bias + (long long)m * NBB + (l == 0 ? BB1 : l == 1 ? BB2 : l == 2 ? BB3 : BB4);
          if (l < 3) {
            unsigned char* hrow = sm + sl * H_BYTES + (r >> 3) * 4096 + (r & 7) * 16;
            // software pipeline over this warp's 8 chunks: the TMEM load and the biases of
            // chunk i + 1 are in flight while chunk i is evaluated
            uint32_t ra[16], rb[16];
            float4 ba[4], bb[4];
            umma::tmem_ld16_issue(trow + half * 16, ra);
#pragma unroll
            for (int j = 0; j < 4; ++j) ba[j] = __ldg(reinterpret_cast<const float4*>(bias + half * 16) + j);
#pragma unroll
            for (int it = 0; it < 8; ++it) {
              const int c16 = half + 2 * it;
              uint32_t (&cur)[16] = (it & 1) ? rb : ra;
              uint32_t (&nxt)[16] = (it & 1) ? ra : rb;
              float4 (&bc)[4] = (it & 1) ? bb : ba;
              float4 (&bn)[4] = (it & 1) ? ba : bb;
              umma::tmem_ld_wait(cur);
              if (it < 7) {
                umma::tmem_ld16_issue(trow + (c16 + 2) * 16, nxt);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  bn[j] = __ldg(reinterpret_cast<const float4*>(bias + (c16 + 2) * 16) + j);
              }
              uint32_t pk[8];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float4 b = bc[j];
                const float2 s0 = __fadd2_rn(make_float2(__uint_as_float(cur[4 * j]),
                                                         __uint_as_float(cur[4 * j + 1])),
                                             make_float2(b.x, b.y));
                const float2 s1 = __fadd2_rn(make_float2(__uint_as_float(cur[4 * j + 2]),
                                                         __uint_as_float(cur[4 * j + 3])),
                                             make_float2(b.z, b.w));
                const float2 g0 = gelu_f2(s0), g1 = gelu_f2(s1);
                const __nv_bfloat162 h0 = __floats2bfloat162_rn(g0.x, g0.y);
                const __nv_bfloat162 h1 = __floats2bfloat162_rn(g1.x, g1.y);
                pk[2 * j] = *reinterpret_cast<const uint32_t*>(&h0);
                pk[2 * j + 1] = *reinterpret_cast<const uint32_t*>(&h1);
              }
              *reinterpret_cast<uint4*>(hrow + (c16 * 2) * 128) =
                  make_uint4(pk[0], pk[1], pk[2], pk[3]);
              *reinterpret_cast<uint4*>(hrow + (c16 * 2 + 1) * 128) =
                  make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            umma::fence_proxy_async();  // H is read next by the tensor cores (async proxy)
          } else if (half == 0) {
            uint32_t rv[16];
            umma::tmem_ld16(trow, rv);
            if (grow < f.B) {
              float* yo = f.y + ((long long)m * f.ystride + grow) * 3;
#pragma unroll
              for (int j = 0; j < 3; ++j)
                yo[j] = fmaf(__uint_as_float(rv[j]) + __ldg(bias + j), __ldg(f.ystat + 3 + j),
                             __ldg(f.ystat + j));
            }
          }
          umma::fence_before();
          umma::mbar_arrive(&hready[sl]);
          ++J;
        }
    }
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();  // the producer lane joins the rest of its warp before the collective free
    umma::fence_after();
    umma::tmem_dealloc<512>(tbase);
  }
}

}  // namespace mlp
}  // namespace ens

using namespace ens;
using namespace ens::mlp;

// ============================================================================ the C ABI
struct ens_mlp {
  int E;
  long long bmax;
  int splits_max;
  Box box;
  float* p;       // [E][NP]
  float* am;      // [E][NP]
  float* av;      // [E][NP]
  float* g;       // [NP] gradient of the last ens_mlp_grad
  bf16* wb;       // [E][NWB]
  float* bb;      // [E][NBB]
  float* ystat;   // [6]: y_mean[3], y_std[3]
  float* one3;    // [6]: ones[3], zeros[3] (identity affine for training)
  bf16* xn;       // [bmax][16]
  float* z[3];    // [bmax][256]
  bf16* h[3];     // [bmax][256]
  float* z4;      // [bmax][16]
  bf16* dz4;      // [bmax][16]
  bf16* dz[2];    // [bmax][256]
  float* part;    // [splits_max][256][256]
  bf16* wp;       // [E][fused::NWP] weights packed for the fused forward
  bf16* xt;       // [bmax / 128][2048] tiled normalised inputs of the fused forward
  int num_sms;
  double* loss;
  int* err;
  void* block;    // single allocation holding everything above
};

namespace {

int mfail(int code, const char* msg) { return set_last_error(code, msg); }

cudaError_t gemm(const GemmArgs& g0, int splits, cudaStream_t s) {
  GemmArgs g = g0;
  if (g.k_chunk <= 0) g.k_chunk = g.K;
  const dim3 grid((g.M + BM - 1) / BM, 1, splits);
  cudaError_t e;
  if (g.N <= 16) {
    e = cudaFuncSetAttribute(k_gemm<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Tile<16>::SMEM);
    if (e != cudaSuccess) return e;
    k_gemm<16><<<grid, NTHREADS, Tile<16>::SMEM, s>>>(g);
  } else {
    e = cudaFuncSetAttribute(k_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Tile<256>::SMEM);
    if (e != cudaSuccess) return e;
    dim3 gr = grid;
    gr.y = (g.N + 255) / 256;
    k_gemm<256><<<gr, NTHREADS, Tile<256>::SMEM, s>>>(g);
  }
  return cudaGetLastError();
}

GemmArgs gemm_args(const ens_mlp* m) {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.err = m->err;
  return g;
}

unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// forward of one member on rows [0, B) of the workspace (x already normalised into xn);
// keep = store the pre-activations for the backward pass; y (if not null) gets the
// de-standardised output [B][3]
cudaError_t forward_member(ens_mlp* m, int e, long long B, bool keep, float* y, long long ldy,
                           cudaStream_t s) {
  const bf16* W = m->wb + (long long)e * NWB;
  const float* bias = m->bb + (long long)e * NBB;
  const bf16* in = m->xn;
  long long ldin = PAD_IN;
  const long long woff[3] = {WB1, WB2, WB3};
  const long long boff[3] = {BB1, BB2, BB3};
  for (int l = 0; l < 3; ++l) {
    GemmArgs g = gemm_args(m);
    g.M = (int)B;
    g.N = HID;
    g.K = l == 0 ? PAD_IN : HID;
    g.A = in;
    g.lda = ldin;
    g.B = W + woff[l];
    g.ldb = l == 0 ? PAD_IN : HID;
    g.epi = EPI_GELU_FWD;
    g.bias = bias + boff[l];
    g.out_f32 = keep ? m->z[l] : nullptr;
    g.ldo = HID;
    g.out_bf16 = m->h[l];
    g.ldob = HID;
    cudaError_t err = gemm(g, 1, s);
    if (err != cudaSuccess) return err;
    in = m->h[l];
    ldin = HID;
  }
  GemmArgs g = gemm_args(m);
  g.M = (int)B;
  g.N = y ? 3 : PAD_OUT;
  g.K = HID;
  g.A = m->h[2];
  g.lda = HID;
  g.B = W + WB4;
  g.ldb = HID;
  g.epi = EPI_AFFINE;
  g.bias = bias + BB4;
  g.scale = y ? m->ystat + 3 : nullptr;
  g.shift = y ? m->ystat : nullptr;
  g.out_f32 = y ? y : m->z4;
  g.ldo = y ? ldy : PAD_OUT;
  return gemm(g, 1, s);
}

// weight gradient dW = dZ^T H over the batch (both operands MN-major), split over K
cudaError_t wgrad(ens_mlp* m, long long B, const bf16* dz, int ldz, int Mrows, const bf16* h,
                  int ldh, int Ncols, float* out, int out_rows, int out_cols, cudaStream_t s) {
  int chunk = (int)std::max<long long>(BK, ((B + m->splits_max - 1) / m->splits_max + BK - 1) /
                                               BK * BK);
  const int splits = (int)((B + chunk - 1) / chunk);
  GemmArgs g = gemm_args(m);
  g.M = Mrows;
  g.N = Ncols;
  g.K = (int)B;
  g.A = dz;
  g.lda = ldz;
  g.a_mn = 1;
  g.B = h;
  g.ldb = ldh;
  g.b_mn = 1;
  g.epi = EPI_PARTIAL;
  g.out_f32 = m->part;
  g.ldo = Ncols;
  g.split_stride = (long long)Mrows * Ncols;
  g.k_chunk = chunk;
  cudaError_t e = gemm(g, splits, s);
  if (e != cudaSuccess) return e;
  const long long n = (long long)out_rows * out_cols;
  k_reduce<<<blocks_for(n), 256, 0, s>>>(splits, (long long)Mrows * Ncols, out_rows, out_cols,
                                         Ncols, m->part, out, out_cols);
  return cudaGetLastError();
}

cudaError_t bias_grad(ens_mlp* m, long long B, const bf16* dz, int ld, int ncols, float* out,
                      cudaStream_t s) {
  const long long chunk = 256;
  const int nchunk = (int)((B + chunk - 1) / chunk);
  // the partial column sums reuse the split-K buffer (after the weight gradient is reduced)
  k_colsum<<<dim3((ncols + 255) / 256, nchunk), 256, 0, s>>>(B, ncols, ld, dz, chunk, m->part);
  k_reduce<<<blocks_for(ncols), 256, 0, s>>>(nchunk, ncols, 1, ncols, ncols, m->part, out, ncols);
  return cudaGetLastError();
}

Box make_box(const double* box) {
  Box b;
  for (int c = 0; c < 6; ++c) {
    b.lo[c] = (float)box[2 * c];
    b.hi[c] = (float)box[2 * c + 1];
    b.inv[c] = (float)(2.0 / (box[2 * c + 1] - box[2 * c]));
  }
  return b;
}

}  // namespace

extern "C" {

long long ens_mlp_n_params(void) { return NP; }

int ens_mlp_create(ens_mlp** out, int members, long long batch_max, const double* box,
                   unsigned long long seed, void* cuda_stream) {
  if (!out) return mfail(ENS_EINVAL, "null output pointer");
  *out = nullptr;
  if (members < 1 || members > 16) return mfail(ENS_EINVAL, "members must be in [1, 16]");
  if (batch_max < 128 || batch_max > (1LL << 24) || batch_max % 128)
    return mfail(ENS_EINVAL, "batch_max must be a multiple of 128 in [128, 2^24]");
  if (!box) return mfail(ENS_EINVAL, "null box");
  for (int c = 0; c < 6; ++c)
    if (!(box[2 * c + 1] > box[2 * c]) || !std::isfinite(box[2 * c]) ||
        !std::isfinite(box[2 * c + 1]))
      return mfail(ENS_EINVAL, "box must have finite lo < hi in every input");
  ens_mlp* m = new ens_mlp();
  std::memset(m, 0, sizeof(*m));
  m->E = members;
  m->bmax = batch_max;
  m->splits_max = 64;
  m->box = make_box(box);
  const long long E = members, Bm = batch_max;
  auto up = [](long long x) { return (x + 255) & ~255LL; };
  long long off = 0;
  long long o_p = off; off += up(4 * E * NP);
  long long o_am = off; off += up(4 * E * NP);
  long long o_av = off; off += up(4 * E * NP);
  long long o_g = off; off += up(4 * NP);
  long long o_wb = off; off += up(2 * E * NWB);
  long long o_bb = off; off += up(4 * E * NBB);
  long long o_ys = off; off += up(4 * 6);
  long long o_one = off; off += up(4 * 6);
  long long o_xn = off; off += up(2 * Bm * PAD_IN);
  long long o_z[3], o_h[3];
  for (int l = 0; l < 3; ++l) { o_z[l] = off; off += up(4 * Bm * HID); }
  for (int l = 0; l < 3; ++l) { o_h[l] = off; off += up(2 * Bm * HID); }
  long long o_z4 = off; off += up(4 * Bm * PAD_OUT);
  long long o_dz4 = off; off += up(2 * Bm * PAD_OUT);
  long long o_dz[2];
  for (int l = 0; l < 2; ++l) { o_dz[l] = off; off += up(2 * Bm * HID); }
  const long long part_elems = std::max<long long>((long long)m->splits_max * HID * HID,
                                                   (Bm / 256 + 1) * HID);
  long long o_part = off; off += up(4 * part_elems);
  long long o_wp = off; off += up(2 * E * fused::NWP);
  long long o_xt = off; off += up(2 * Bm * PAD_IN);
  long long o_loss = off; off += up(8);
  long long o_err = off; off += up(4);
  if (cudaMalloc(&m->block, off) != cudaSuccess) {
    delete m;
    return mfail(ENS_ENOMEM, "surrogate network memory");
  }
  char* b = (char*)m->block;
  m->p = (float*)(b + o_p);
  m->am = (float*)(b + o_am);
  m->av = (float*)(b + o_av);
  m->g = (float*)(b + o_g);
  m->wb = (bf16*)(b + o_wb);
  m->bb = (float*)(b + o_bb);
  m->ystat = (float*)(b + o_ys);
  m->one3 = (float*)(b + o_one);
  m->xn = (bf16*)(b + o_xn);
  for (int l = 0; l < 3; ++l) {
    m->z[l] = (float*)(b + o_z[l]);
    m->h[l] = (bf16*)(b + o_h[l]);
  }
  m->z4 = (float*)(b + o_z4);
  m->dz4 = (bf16*)(b + o_dz4);
  for (int l = 0; l < 2; ++l) m->dz[l] = (bf16*)(b + o_dz[l]);
  m->part = (float*)(b + o_part);
  m->wp = (bf16*)(b + o_wp);
  m->xt = (bf16*)(b + o_xt);
  m->loss = (double*)(b + o_loss);
  m->err = (int*)(b + o_err);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    m->num_sms = 1;
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const float ys[6] = {0.f, 0.f, 0.f, 1.f, 1.f, 1.f};
  cudaError_t e = cudaMemcpyAsync(m->ystat, ys, sizeof(ys), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->one3, ys, sizeof(ys), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->am, 0, 4 * E * NP, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->av, 0, 4 * E * NP, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, 4, s);
  for (int k = 0; k < members && e == cudaSuccess; ++k) {
    k_init<<<blocks_for(NP), 256, 0, s>>>(NP, k, seed, m->p + k * NP);
    k_refresh<<<blocks_for(NWB), 256, 0, s>>>(m->p + k * NP, m->wb + k * NWB, m->bb + k * NBB);
    k_pack<<<blocks_for(fused::NWP), 256, 0, s>>>(m->p + k * NP, m->wp + k * fused::NWP);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host arrays above are stack memory
  if (e != cudaSuccess) {
    cudaFree(m->block);
    delete m;
    return mfail(ENS_ECUDA, cudaGetErrorString(e));
  }
  *out = m;
  return ENS_OK;
}

int ens_mlp_destroy(ens_mlp* m) {
  if (!m) return ENS_OK;
  cudaDeviceSynchronize();
  cudaFree(m->block);
  delete m;
  return ENS_OK;
}

int ens_mlp_set_scaling(ens_mlp* m, const double* y_mean, const double* y_std, void* stream) {
  if (!m || !y_mean || !y_std) return mfail(ENS_EINVAL, "null argument");
  float ys[6];
  for (int j = 0; j < 3; ++j) {
    if (!(y_std[j] > 0) || !std::isfinite(y_std[j]) || !std::isfinite(y_mean[j]))
      return mfail(ENS_EINVAL, "y_std must be finite and > 0");
    ys[j] = (float)y_mean[j];
    ys[3 + j] = (float)y_std[j];
  }
  cudaError_t e = cudaMemcpyAsync(m->ystat, ys, sizeof(ys), cudaMemcpyHostToDevice,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_params(ens_mlp* m, int member, float* get, const float* set, void* stream) {
  if (!m) return mfail(ENS_EINVAL, "null network");
  if (member < 0 || member >= m->E) return mfail(ENS_EINVAL, "member out of range");
  cudaStream_t s = (cudaStream_t)stream;
  float* p = m->p + (long long)member * NP;
  cudaError_t e = cudaSuccess;
  if (get) e = cudaMemcpyAsync(get, p, 4 * NP, cudaMemcpyDeviceToDevice, s);
  if (set && e == cudaSuccess) {
    e = cudaMemcpyAsync(p, set, 4 * NP, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
      k_refresh<<<blocks_for(NWB), 256, 0, s>>>(p, m->wb + member * NWB, m->bb + member * NBB);
      k_pack<<<blocks_for(fused::NWP), 256, 0, s>>>(p, m->wp + member * fused::NWP);
      e = cudaGetLastError();
    }
  }
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_grad(ens_mlp* m, int member, long long B, const float* x, const float* y,
                 const long long* idx, float* grad, double* loss, void* stream) {
  if (!m) return mfail(ENS_EINVAL, "null network");
  if (member < 0 || member >= m->E) return mfail(ENS_EINVAL, "member out of range");
  if (B < 1 || B > m->bmax) return mfail(ENS_EINVAL, "B must be in [1, batch_max]");
  if (!x || !y) return mfail(ENS_EINVAL, "null array");
  cudaStream_t s = (cudaStream_t)stream;
  const int e_ = member;
  const bf16* W = m->wb + (long long)e_ * NWB;
  cudaError_t e = cudaMemsetAsync(m->loss, 0, 8, s);
  k_input<<<blocks_for(B * PAD_IN), 256, 0, s>>>(B, x, idx, m->box, m->xn);
  if (e == cudaSuccess) e = forward_member(m, e_, B, true, nullptr, 0, s);
  if (e == cudaSuccess) {
    k_loss<<<blocks_for(B * PAD_OUT), 256, 0, s>>>(B, m->z4, y, idx, m->ystat, m->ystat + 3,
                                                   m->dz4, m->loss);
    e = cudaGetLastError();
  }
  float* G = m->g;
  // layer 4: dW4 = dZ4^T H3 (rows 0..2), db4, dZ3 = (dZ4 W4) * gelu'(Z3)
  if (e == cudaSuccess) e = wgrad(m, B, m->dz4, PAD_OUT, PAD_OUT, m->h[2], HID, HID,
                                  G + OFF_W4, 3, HID, s);
  if (e == cudaSuccess) e = bias_grad(m, B, m->dz4, PAD_OUT, 3, G + OFF_B4, s);
  const bf16* dzl = m->dz4;
  int lddz = PAD_OUT;
  const long long woff[4] = {WB1, WB2, WB3, WB4};
  const long long goffW[3] = {OFF_W1, OFF_W2, OFF_W3};
  const long long goffB[3] = {OFF_B1, OFF_B2, OFF_B3};
  for (int l = 2; l >= 0 && e == cudaSuccess; --l) {
    // dZ_l = (dZ_{l+1} W_{l+1}) * gelu'(Z_l): A = dZ_{l+1} (K-major), B(n,k) = W_{l+1}[k][n]
    bf16* dzn = m->dz[l & 1];
    GemmArgs g = gemm_args(m);
    g.M = (int)B;
    g.N = HID;
    g.K = lddz;
    g.A = dzl;
    g.lda = lddz;
    g.B = W + woff[l + 1];
    g.ldb = HID;
    g.b_mn = 1;
    g.epi = EPI_GELU_BWD;
    g.aux = m->z[l];
    g.ldaux = HID;
    g.out_bf16 = dzn;
    g.ldob = HID;
    e = gemm(g, 1, s);
    // dW_l = dZ_l^T H_{l-1}, db_l
    const bf16* hin = l == 0 ? m->xn : m->h[l - 1];
    const int ldh = l == 0 ? PAD_IN : HID;
    const int ncol = l == 0 ? PAD_IN : HID;
    if (e == cudaSuccess)
      e = wgrad(m, B, dzn, HID, HID, hin, ldh, ncol, G + goffW[l], HID, l == 0 ? 6 : HID, s);
    if (e == cudaSuccess) e = bias_grad(m, B, dzn, HID, HID, G + goffB[l], s);
    dzl = dzn;
    lddz = HID;
  }
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, G, 4 * NP, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, m->loss, 8, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_adam(ens_mlp* m, int member, float lr, int t, void* stream) {
  if (!m) return mfail(ENS_EINVAL, "null network");
  if (member < 0 || member >= m->E) return mfail(ENS_EINVAL, "member out of range");
  if (t < 1 || !(lr >= 0)) return mfail(ENS_EINVAL, "t must be >= 1 and lr >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, t)), c2 = (float)(1.0 - std::pow(0.999, t));
  const long long o = (long long)member * NP;
  k_adam<<<blocks_for(NP), 256, 0, s>>>(NP, m->p + o, m->g, m->am + o, m->av + o, lr, b1, b2,
                                        1e-8f, c1, c2);
  k_refresh<<<blocks_for(NWB), 256, 0, s>>>(m->p + o, m->wb + member * NWB, m->bb + member * NBB);
  k_pack<<<blocks_for(fused::NWP), 256, 0, s>>>(m->p + o, m->wp + member * fused::NWP);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_forward(ens_mlp* m, int member, long long B, const float* x, float* y, int flags,
                    void* stream) {
  if (!m) return mfail(ENS_EINVAL, "null network");
  if (member < -1 || member >= m->E) return mfail(ENS_EINVAL, "member out of range");
  if (B < 0) return mfail(ENS_EINVAL, "B < 0");
  if (flags & ~ENS_MLP_LAYERWISE) return mfail(ENS_EINVAL, "unknown flags");
  if (B == 0) return ENS_OK;
  if (!x || !y) return mfail(ENS_EINVAL, "null array");
  cudaStream_t s = (cudaStream_t)stream;
  const int e0 = member < 0 ? 0 : member, e1 = member < 0 ? m->E : member + 1;
  cudaError_t e = cudaSuccess;
  if (!(flags & ENS_MLP_LAYERWISE)) {
    e = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             fused::SMEM);
    for (long long b0 = 0; b0 < B && e == cudaSuccess; b0 += m->bmax) {
      const long long nb = std::min(m->bmax, B - b0);
      const long long rows = (nb + 127) / 128 * 128;
      k_input_tiled<<<blocks_for(rows * PAD_IN), 256, 0, s>>>(nb, rows, x + b0 * 6, m->box, m->xt);
      FusedArgs f;
      f.B = nb;
      f.ystride = B;
      f.ntiles = (int)(rows / 128);
      f.E = e1 - e0;
      f.xt = m->xt;
      f.wp = m->wp + (long long)e0 * fused::NWP;
      f.bias = m->bb + (long long)e0 * NBB;
      f.ystat = m->ystat;
      f.y = y + b0 * 3;
      f.err = m->err;
      const int grid = std::max(1, std::min((f.ntiles + 1) / 2, m->num_sms));
      k_mlp_fused<<<grid, fused::NT, fused::SMEM, s>>>(f);
      e = cudaGetLastError();
    }
    return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
  }
  for (long long b0 = 0; b0 < B && e == cudaSuccess; b0 += m->bmax) {
    const long long nb = std::min(m->bmax, B - b0);
    k_input<<<blocks_for(nb * PAD_IN), 256, 0, s>>>(nb, x + b0 * 6, nullptr, m->box, m->xn);
    e = cudaGetLastError();
    for (int k = e0; k < e1 && e == cudaSuccess; ++k)
      e = forward_member(m, k, nb, false, y + ((long long)(k - e0) * B + b0) * 3, 3, s);
  }
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_gate(ens_mlp* m, long long B, const float* x, const float* y_members, float tau,
                 float* y_mean, float* spread, unsigned char* fallback, unsigned long long* n_fallback,
                 long long* fb_index, float* fb_params, float* fb_u0, float* fb_tspan, double t0,
                 double t1, void* stream) {
  if (!m) return mfail(ENS_EINVAL, "null network");
  if (B < 0) return mfail(ENS_EINVAL, "B < 0");
  if (B == 0) return ENS_OK;
  if (!x || !y_members || !fallback) return mfail(ENS_EINVAL, "null array");
  if (fb_index && (!fb_params || !fb_u0 || !fb_tspan || !n_fallback))
    return mfail(ENS_EINVAL, "compaction needs fb_params, fb_u0, fb_tspan and n_fallback");
  Compact cp{fb_index, fb_params, fb_u0, fb_tspan, (float)t0, (float)t1};
  k_gate<<<blocks_for(B), 256, 0, (cudaStream_t)stream>>>(B, m->E, x, y_members, m->box, tau,
                                                          y_mean, spread, fallback, n_fallback, cp);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_scatter(long long n, const long long* fb_index, const float* u, float* y,
                    void* stream) {
  if (n < 0) return mfail(ENS_EINVAL, "n < 0");
  if (n == 0) return ENS_OK;
  if (!fb_index || !u || !y) return mfail(ENS_EINVAL, "null array");
  k_scatter<<<blocks_for(n * 3), 256, 0, (cudaStream_t)stream>>>(n, fb_index, u, y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_activation(int which, long long n, const float* z, float* out, void* stream) {
  if (which != 0 && which != 1) return mfail(ENS_EINVAL, "which must be 0 (gelu) or 1 (gelu')");
  if (n < 0) return mfail(ENS_EINVAL, "n < 0");
  if (n == 0) return ENS_OK;
  if (!z || !out) return mfail(ENS_EINVAL, "null array");
  k_activation<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(which, n, z, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ENS_OK : mfail(ENS_ECUDA, cudaGetErrorString(e));
}

int ens_mlp_check(ens_mlp* m, void* stream) {
  if (!m) return mfail(ENS_EINVAL, "null network");
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, m->err, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return mfail(ENS_ECUDA, cudaGetErrorString(e));
  if (h) return mfail(ENS_ECUDA, "a tensor-core wait timed out (results invalid)");
  return ENS_OK;
}

}  // extern "C"
