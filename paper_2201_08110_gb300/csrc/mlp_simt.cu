// mlp_simt.cu -- grouped matrix products of the atomic networks on the FP32
// SIMT pipes (the plain FP32 path), with the networks' epilogues fused.
//
// Every product is D[M, N] = A[M, K] * B[N, K]^T with A and B K-major; the
// problem list covers all elements and ensemble members of one layer, and a
// tile table flattens their output tiles into one launch.  Tiles are 64 x 64,
// 256 threads, 4 x 4 outputs per thread, K in steps of 16 staged through
// shared memory.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

template <typename T> __device__ __forceinline__ float ld_f(const T* p);
template <> __device__ __forceinline__ float ld_f<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_f<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <> __device__ __forceinline__ float ld_f<__half>(const __half* p) { return __half2float(*p); }
template <typename T> __device__ __forceinline__ void st_f(T* p, float v);
template <> __device__ __forceinline__ void st_f<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void st_f<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ void st_f<__half>(__half* p, float v) { *p = __float2half_rn(v); }

constexpr int BM = 64, BN = 64, BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_simt(const GemmProblem* __restrict__ probs,
                                                   const GemmTile* __restrict__ tiles) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmProblem P = probs[tl.problem];
  const T* __restrict__ A = static_cast<const T*>(P.A);
  const T* __restrict__ B = static_cast<const T*>(P.B);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < P.K; k0 += BK) {
#pragma unroll
    for (int it = 0; it < (BM * BK) / 256; ++it) {
      const int idx = threadIdx.x + it * 256;
      const int r = idx / BK, kk = idx % BK;
      const int gm = tl.m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < P.M && gk < P.K) ? ld_f(A + (size_t)gm * P.lda + gk) : 0.f;
      const int gn = tl.n0 + r;
      Bs[kk][r] = (gn < P.N && gk < P.K) ? ld_f(B + (size_t)gn * P.ldb + gk) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = tl.m0 + ty * 4 + i;
    if (m >= P.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = tl.n0 + tx * 4 + j;
      if (n >= P.N) continue;
      const float v = acc[i][j];
      switch (P.epi) {
        case (int)Epi::BiasCelu: {
          const float z = v + P.bias[n];
          // alpha expm1(z / alpha): exp(z / alpha) - 1 would cancel for small |z|
          const float h = z > 0.f ? z : 0.1f * expm1f(fminf(z, 0.f) * 10.f);
          st_f(static_cast<T*>(P.D) + (size_t)m * P.ldd + n, h);
          break;
        }
        case (int)Epi::Bias:
          static_cast<float*>(P.D)[(size_t)m * P.ldd + n] = v + P.bias[n];
          break;
        case (int)Epi::DCelu: {
          T* d = static_cast<T*>(P.D) + (size_t)m * P.ldd + n;
          const float h = ld_f(d);
          st_f(d, v * (h > 0.f ? 1.f : fmaf(10.f, h, 1.f)));
          break;
        }
        default:
          static_cast<float*>(P.D)[(size_t)m * P.ldd + n] = v;
          break;
      }
    }
  }
}

}  // namespace

void launch_gemm_simt_typed(const GemmProblem* probs, const GemmTile* tiles, int n_tiles, Prec p,
                            cudaStream_t s) {
  if (n_tiles <= 0) return;
  switch (p) {
    case Prec::F32: k_gemm_simt<float><<<n_tiles, 256, 0, s>>>(probs, tiles); break;
    case Prec::BF16: k_gemm_simt<__nv_bfloat16><<<n_tiles, 256, 0, s>>>(probs, tiles); break;
    case Prec::F16: k_gemm_simt<__half><<<n_tiles, 256, 0, s>>>(probs, tiles); break;
  }
}

void launch_gemm_simt(const GemmProblem* probs, const GemmTile* tiles, int n_tiles, cudaStream_t s) {
  launch_gemm_simt_typed(probs, tiles, n_tiles, Prec::F32, s);
}

}  // namespace nnp
