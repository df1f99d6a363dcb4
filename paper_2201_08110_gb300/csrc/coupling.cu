// coupling.cu -- the NNP-MM coupling term of the hybrid potential (Eq. 4, the
// mechanical-embedding scheme of Sec. 2):
//
//   V_NNP-MM = sum_{i in NNP} sum_{j in MM} ke q_i q_j / r_ij
//                 + 4 eps_ij ((sigma_ij / r_ij)^12 - (sigma_ij / r_ij)^6)
//   sigma_ij = (sigma_i + sigma_j) / 2,  eps_ij = sqrt(eps_i eps_j)
//
// over every NNP-MM pair (no cutoff, no periodic images, as the equation is
// written), with its forces added into the callers' FP64 force buffers.
//
// One thread owns kCplJ MM atoms and keeps their forces in registers; the NNP
// atoms (a ligand: at most NNP_COUPLING_MAX_NNP) sit in shared memory with their charge
// pre-multiplied by ke, half their sigma and twice the square root of their
// eps, so a pair needs one reciprocal square root and no division: with
// s6 = (sigma_ij / r)^6,
//   V_LJ = (2 sqrt eps_i)(2 sqrt eps_j) s6 (s6 - 1),
//   -dV/dr / r = (V_C + 4 eps_ij s6 (12 s6 - 6)) / r^2.
// Pair arithmetic is FP32.  Each NNP atom's force is summed over the warp by
// shuffles into the warp's own row in shared memory, over the CTA's warps in
// FP64 in a fixed order and over CTAs with FP64 atomics; each thread's energy
// is summed in FP32 over its pairs and from there in FP64.  Within a CTA the
// order of every sum is fixed.
#include <cuda_runtime.h>

#include "../../include/nnp.h"

namespace {

constexpr int kCplThreads = 128;
constexpr int kCplWarps = kCplThreads / 32;
constexpr int kCplJ = 2;  // MM atoms per thread

__global__ void __launch_bounds__(kCplThreads)
    k_coupling(const float* __restrict__ xn, const float* __restrict__ qn,
               const float* __restrict__ sn, const float* __restrict__ en, int n_nnp,
               const float* __restrict__ xm, const float* __restrict__ qm,
               const float* __restrict__ sm, const float* __restrict__ em, int n_mm, float ke,
               double* __restrict__ energy, double* __restrict__ f_nnp, double* __restrict__ f_mm) {
  extern __shared__ float4 sh[];
  float4* nx = sh;                                          // [n_nnp] x, y, z, ke q
  float2* np = reinterpret_cast<float2*>(nx + n_nnp);       // [n_nnp] sigma / 2, 2 sqrt(eps)
  float* nf = reinterpret_cast<float*>(np + n_nnp);         // [warps][n_nnp][3] forces per warp
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < n_nnp; t += blockDim.x) {
    nx[t] = make_float4(xn[3 * t], xn[3 * t + 1], xn[3 * t + 2], ke * qn[t]);
    np[t] = make_float2(0.5f * sn[t], 2.f * sqrtf(en[t]));
  }
  __syncthreads();
  float* nf_w = nf + (size_t)warp * 3 * n_nnp;

  float xj[kCplJ][3], qj[kCplJ], hsj[kCplJ], sej[kCplJ], fj[kCplJ][3];
  bool vj[kCplJ];
#pragma unroll
  for (int u = 0; u < kCplJ; ++u) {
    const int j = blockIdx.x * (kCplThreads * kCplJ) + u * kCplThreads + threadIdx.x;
    vj[u] = j < n_mm;
    const int jj = vj[u] ? j : 0;
    xj[u][0] = xm[3 * jj];
    xj[u][1] = xm[3 * jj + 1];
    xj[u][2] = xm[3 * jj + 2];
    qj[u] = qm[jj];
    hsj[u] = 0.5f * sm[jj];
    sej[u] = 2.f * sqrtf(em[jj]);
    fj[u][0] = fj[u][1] = fj[u][2] = 0.f;
  }

  float e_thr = 0.f;
  for (int i = 0; i < n_nnp; ++i) {
    const float4 a = nx[i];
    const float2 p = np[i];
    float fix = 0.f, fiy = 0.f, fiz = 0.f;
#pragma unroll
    for (int u = 0; u < kCplJ; ++u) {
      if (!vj[u]) continue;
      const float dx = xj[u][0] - a.x, dy = xj[u][1] - a.y, dz = xj[u][2] - a.z;  // i -> j
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float ir = rsqrtf(r2);
      const float ir2 = ir * ir;
      const float sig = p.x + hsj[u];
      const float eps4 = p.y * sej[u];  // 4 eps_ij
      const float s2 = sig * sig * ir2;
      const float s6 = s2 * s2 * s2;
      const float vc = a.w * qj[u] * ir;
      e_thr += fmaf(eps4 * s6, s6 - 1.f, vc);
      const float fs = fmaf(eps4 * s6, fmaf(12.f, s6, -6.f), vc) * ir2;  // -dV/dr / r
      fj[u][0] = fmaf(fs, dx, fj[u][0]);
      fj[u][1] = fmaf(fs, dy, fj[u][1]);
      fj[u][2] = fmaf(fs, dz, fj[u][2]);
      fix = fmaf(-fs, dx, fix);
      fiy = fmaf(-fs, dy, fiy);
      fiz = fmaf(-fs, dz, fiz);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      fix += __shfl_xor_sync(FULL, fix, o);
      fiy += __shfl_xor_sync(FULL, fiy, o);
      fiz += __shfl_xor_sync(FULL, fiz, o);
    }
    if (lane == 0) {  // every (warp, i) written once
      nf_w[3 * i] = fix;
      nf_w[3 * i + 1] = fiy;
      nf_w[3 * i + 2] = fiz;
    }
  }

#pragma unroll
  for (int u = 0; u < kCplJ; ++u) {
    if (!vj[u]) continue;
    const size_t j = (size_t)blockIdx.x * (kCplThreads * kCplJ) + u * kCplThreads + threadIdx.x;
    f_mm[3 * j] += (double)fj[u][0];  // one thread per MM atom: no other writer
    f_mm[3 * j + 1] += (double)fj[u][1];
    f_mm[3 * j + 2] += (double)fj[u][2];
  }
  double e = (double)e_thr;
#pragma unroll
  for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
  if (lane == 0) atomicAdd(energy, e);
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * n_nnp; t += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < kCplWarps; ++w) sum += (double)nf[(size_t)w * 3 * n_nnp + t];
    atomicAdd(f_nnp + t, sum);
  }
}

}  // namespace

extern "C" nnp_status nnp_mm_coupling(const float* nnp_positions_dev, const float* nnp_charges_dev,
                                      const float* nnp_sigma_dev, const float* nnp_epsilon_dev,
                                      int32_t n_nnp, const float* mm_positions_dev,
                                      const float* mm_charges_dev, const float* mm_sigma_dev,
                                      const float* mm_epsilon_dev, int32_t n_mm, double coulomb_k,
                                      double* energy_dev, double* nnp_forces_dev,
                                      double* mm_forces_dev, void* stream) {
  if (n_nnp < 0 || n_mm < 0) return NNP_ERR_ARG;
  if (n_nnp > NNP_COUPLING_MAX_NNP) return NNP_ERR_TOO_LARGE;
  if (n_nnp == 0 || n_mm == 0) return NNP_OK;
  if (!nnp_positions_dev || !nnp_charges_dev || !nnp_sigma_dev || !nnp_epsilon_dev ||
      !mm_positions_dev || !mm_charges_dev || !mm_sigma_dev || !mm_epsilon_dev || !energy_dev ||
      !nnp_forces_dev || !mm_forces_dev)
    return NNP_ERR_ARG;
  const int per_cta = kCplThreads * kCplJ;
  const int grid = (n_mm + per_cta - 1) / per_cta;
  const size_t smem = (size_t)n_nnp * (sizeof(float4) + sizeof(float2) + kCplWarps * 3 * sizeof(float));
  k_coupling<<<grid, kCplThreads, smem, static_cast<cudaStream_t>(stream)>>>(
      nnp_positions_dev, nnp_charges_dev, nnp_sigma_dev, nnp_epsilon_dev, n_nnp, mm_positions_dev,
      mm_charges_dev, mm_sigma_dev, mm_epsilon_dev, n_mm, (float)coulomb_k, energy_dev,
      nnp_forces_dev, mm_forces_dev);
  return cudaGetLastError() == cudaSuccess ? NNP_OK : NNP_ERR_CUDA;
}
