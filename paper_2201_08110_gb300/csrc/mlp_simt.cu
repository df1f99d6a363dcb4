// mlp_simt.cu -- grouped matrix products of the atomic networks on the FP32
// SIMT pipes (the plain FP32 path), with the networks' epilogues fused.
//
// Every product is D[M, N] = A[M, K] * B[N, K]^T with A and B K-major (rows
// and leading dimensions 16-byte aligned, K a multiple of 4); the problem
// list covers all elements and ensemble members of one layer, and a tile
// table flattens their output tiles (simt_tile_m() x simt_tile_n()) into one
// launch.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

// Tiles of BM x BN outputs, 256 threads as 16 x 16, each thread TM x TN
// outputs (rows ty * TM.., columns tx * TN..); K in steps of BK staged
// through shared memory (transposed, k-major, rows padded so the 16-byte
// reads stay aligned), the next step's operands fetched into registers while
// the current one is multiplied (one barrier per step).
constexpr int TM = 8, TN = 4, BK = 16;
constexpr int BM = 16 * TM, BN = 16 * TN;
constexpr int kPadM = BM + 4, kPadN = BN + 4;

__global__ void __launch_bounds__(256, 3) k_gemm_simt(const GemmProblem* __restrict__ probs,
                                                   const GemmTile* __restrict__ tiles) {
  __shared__ __align__(16) float As[2][BK][kPadM];
  __shared__ __align__(16) float Bs[2][BK][kPadN];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmProblem P = probs[tl.problem];
  const float* __restrict__ A = static_cast<const float*>(P.A);
  const float* __restrict__ B = static_cast<const float*>(P.B);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // loader: float4 k4 (of BK / 4) of A rows lr and lr + 64, of B row lr
  const int lr = tid >> 2, k4 = (tid & 3) * 4;
  float4 ra[2], rb;
  auto fetch = [&](int k0) {
    const int gk = k0 + k4;
    const bool kin = gk < P.K;  // K is a multiple of 4
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int gm = tl.m0 + lr + 64 * i;
      ra[i] = (kin && gm < P.M) ? __ldg(reinterpret_cast<const float4*>(A + (size_t)gm * P.lda + gk))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int gn = tl.n0 + lr;
    rb = (kin && gn < P.N) ? __ldg(reinterpret_cast<const float4*>(B + (size_t)gn * P.ldb + gk))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      As[buf][k4 + 0][lr + 64 * i] = ra[i].x;
      As[buf][k4 + 1][lr + 64 * i] = ra[i].y;
      As[buf][k4 + 2][lr + 64 * i] = ra[i].z;
      As[buf][k4 + 3][lr + 64 * i] = ra[i].w;
    }
    Bs[buf][k4 + 0][lr] = rb.x;
    Bs[buf][k4 + 1][lr] = rb.y;
    Bs[buf][k4 + 2][lr] = rb.z;
    Bs[buf][k4 + 3][lr] = rb.w;
  };
  float2 acc[TM][TN / 2];  // columns (2j, 2j + 1) as a pair: packed FP32 products
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);

  fetch(0);
  stage(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < P.K; k0 += BK) {
    const bool more = k0 + BK < P.K;
    if (more) fetch(k0 + BK);  // in flight during this step's products
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * TN]);
      const float av[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float2 bv[TN / 2] = {make_float2(b.x, b.y), make_float2(b.z, b.w)};
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) acc[i][j] = __ffma2_rn(make_float2(av[i], av[i]), bv[j], acc[i][j]);
    }
    if (more) {
      stage(buf ^ 1);  // the other buffer: its readers finished before the last barrier
      __syncthreads();
      buf ^= 1;
    }
  }

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = tl.m0 + ty * TM + i;
    if (m >= P.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = tl.n0 + tx * TN + j;
      if (n >= P.N) continue;
      const float v = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
      float* d = static_cast<float*>(P.D) + (size_t)m * P.ldd + n;
      switch (P.epi) {
        case (int)Epi::BiasCelu: {
          const float z = v + P.bias[n];
          // alpha expm1(z / alpha): exp(z / alpha) - 1 would cancel for small |z|
          *d = z > 0.f ? z : 0.1f * expm1f(fminf(z, 0.f) * 10.f);
          break;
        }
        case (int)Epi::Bias:
          *d = v + P.bias[n];
          break;
        case (int)Epi::DCelu: {
          const float h = *d;
          *d = v * (h > 0.f ? 1.f : fmaf(10.f, h, 1.f));
          break;
        }
        default:
          *d = v;
          break;
      }
    }
  }
}

}  // namespace

int simt_tile_m() { return BM; }
int simt_tile_n() { return BN; }

void launch_gemm_simt(const GemmProblem* probs, const GemmTile* tiles, int n_tiles, cudaStream_t s) {
  if (n_tiles <= 0) return;
  k_gemm_simt<<<n_tiles, 256, 0, s>>>(probs, tiles);
}

}  // namespace nnp
