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
// Work split: a CTA of kCplWarps warps takes kCplJ x 32 MM atoms (lane l owns
// atoms l, l + 32, ... of the CTA's tile, with their forces in registers) and
// warp w takes the NNP atoms w, w + kCplWarps, ...; so a ligand of 60 atoms
// against 60,000 MM atoms runs 469 CTAs of 8 warps (about 25 warps per SM)
// with no atom shared between two threads of a warp.  The NNP atoms (at most
// NNP_COUPLING_MAX_NNP) sit in shared memory with their charge pre-multiplied
// by ke, half their sigma and twice the square root of their eps, so a pair
// needs one reciprocal square root and no division: with s6 = (sigma_ij / r)^6,
//   V_LJ = (2 sqrt eps_i)(2 sqrt eps_j) s6 (s6 - 1),
//   -dV/dr / r = (V_C + 4 eps_ij s6 (12 s6 - 6)) / r^2.
// Pair arithmetic is FP32, and so are the sums inside a cluster (FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU): each NNP
// atom's force is summed over its warp's lanes by shuffles, then by the first
// CTA of a thread-block cluster over the 8 CTAs' shared memory (distributed
// shared memory, in CTA order), and added to the caller's FP64 buffer once
// per cluster: every cluster adds into the same few cache lines, so fewer
// additions there is what bounds the kernel's time.  Each MM atom's force is
// summed over the CTA's 8 warps in a fixed order through shared memory and
// added once (no other CTA touches it); the energy goes like the NNP forces.
// Results differ between calls only by the order of the FP64 additions of the
// clusters.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "../../include/nnp.h"

namespace {

namespace cg = cooperative_groups;

constexpr int kCplWarps = 8;
constexpr int kCplThreads = 32 * kCplWarps;
constexpr int kCplJ = 4;                    // MM atoms per lane
constexpr int kCplTile = 32 * kCplJ;        // MM atoms per CTA
constexpr int kCplCluster = 8;              // CTAs per cluster (the grid is padded to a multiple)

__global__ void __cluster_dims__(kCplCluster, 1, 1) __launch_bounds__(kCplThreads)
    k_coupling(const float* __restrict__ xn, const float* __restrict__ qn,
               const float* __restrict__ sn, const float* __restrict__ en, int n_nnp,
               const float* __restrict__ xm, const float* __restrict__ qm,
               const float* __restrict__ sm, const float* __restrict__ em, int n_mm, float ke,
               double* __restrict__ energy, double* __restrict__ f_nnp, double* __restrict__ f_mm) {
  extern __shared__ float4 sh[];
  float4* nx = sh;                                       // [n_nnp] x, y, z, ke q
  float2* np = reinterpret_cast<float2*>(nx + n_nnp);    // [n_nnp] sigma / 2, 2 sqrt(eps)
  float* mf = reinterpret_cast<float*>(np + n_nnp);      // [warps][tile][3] MM forces per warp
  float* ew = mf + kCplWarps * kCplTile * 3;             // [warps] energies
  float* part = ew + kCplWarps;                          // [3 n_nnp + 1] this CTA's NNP forces, energy
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cg::cluster_group cluster = cg::this_cluster();
  for (int t = threadIdx.x; t < n_nnp; t += blockDim.x) {
    nx[t] = make_float4(xn[3 * t], xn[3 * t + 1], xn[3 * t + 2], ke * qn[t]);
    np[t] = make_float2(0.5f * sn[t], 2.f * sqrtf(en[t]));
  }

  const int tile0 = blockIdx.x * kCplTile;
  float xj[kCplJ][3], qj[kCplJ], hsj[kCplJ], sej[kCplJ], fj[kCplJ][3];
  bool vj[kCplJ];
#pragma unroll
  for (int u = 0; u < kCplJ; ++u) {
    const int j = tile0 + u * 32 + lane;
    vj[u] = j < n_mm;
    const int jj = vj[u] ? j : 0;
    xj[u][0] = xm[3 * jj];
    xj[u][1] = xm[3 * jj + 1];
    xj[u][2] = xm[3 * jj + 2];
    qj[u] = vj[u] ? qm[jj] : 0.f;  // a lane past the end adds nothing
    hsj[u] = 0.5f * sm[jj];
    sej[u] = vj[u] ? 2.f * sqrtf(em[jj]) : 0.f;
    if (!vj[u]) xj[u][0] += 1e3f;  // and stays away from every NNP atom
    fj[u][0] = fj[u][1] = fj[u][2] = 0.f;
  }
  __syncthreads();

  float e_thr = 0.f;
  for (int i = warp; i < n_nnp; i += kCplWarps) {
    const float4 a = nx[i];
    const float2 p = np[i];
    float fix = 0.f, fiy = 0.f, fiz = 0.f;
#pragma unroll
    for (int u = 0; u < kCplJ; ++u) {
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
    if (lane == 0) {  // this CTA's share of NNP atom i: one warp owns it
      part[3 * i] = fix;
      part[3 * i + 1] = fiy;
      part[3 * i + 2] = fiz;
    }
  }
  // MM forces: each warp's partial into shared memory, summed over the warps
#pragma unroll
  for (int u = 0; u < kCplJ; ++u)
#pragma unroll
    for (int d = 0; d < 3; ++d) mf[((size_t)warp * kCplTile + u * 32 + lane) * 3 + d] = fj[u][d];
#pragma unroll
  for (int o = 16; o; o >>= 1) e_thr += __shfl_xor_sync(FULL, e_thr, o);
  if (lane == 0) ew[warp] = e_thr;
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * kCplTile; t += blockDim.x) {
    const int j = tile0 + t / 3;
    if (j >= n_mm) continue;
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < kCplWarps; ++w) sum += mf[(size_t)w * kCplTile * 3 + t];
    f_mm[3 * (size_t)tile0 + t] += (double)sum;  // this CTA alone owns these MM atoms
  }
  if (threadIdx.x == 0) {
    float es = 0.f;
#pragma unroll
    for (int w = 0; w < kCplWarps; ++w) es += ew[w];
    part[3 * n_nnp] = es;
  }
  cluster.sync();  // every CTA's partial sums are written
  if (cluster.block_rank() == 0) {
    for (int t = threadIdx.x; t <= 3 * n_nnp; t += blockDim.x) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < kCplCluster; ++c) s += cluster.map_shared_rank(part, c)[t];
      atomicAdd(t < 3 * n_nnp ? f_nnp + t : energy, (double)s);
    }
  }
  cluster.sync();  // the other CTAs' shared memory stays until the first CTA has read it
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
  const int tiles = (n_mm + kCplTile - 1) / kCplTile;
  const int grid = (tiles + kCplCluster - 1) / kCplCluster * kCplCluster;  // CTAs past n_mm add zeros
  const size_t smem = (size_t)n_nnp * (sizeof(float4) + sizeof(float2)) +
                      ((size_t)kCplWarps * (kCplTile * 3 + 1) + 3 * (size_t)n_nnp + 1) * sizeof(float);
  k_coupling<<<grid, kCplThreads, smem, static_cast<cudaStream_t>(stream)>>>(
      nnp_positions_dev, nnp_charges_dev, nnp_sigma_dev, nnp_epsilon_dev, n_nnp, mm_positions_dev,
      mm_charges_dev, mm_sigma_dev, mm_epsilon_dev, n_mm, (float)coulomb_k, energy_dev,
      nnp_forces_dev, mm_forces_dev);
  return cudaGetLastError() == cudaSuccess ? NNP_OK : NNP_ERR_CUDA;
}
