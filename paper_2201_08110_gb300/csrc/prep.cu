// prep.cu -- batch layout (element sort), position gather, network head,
// per-molecule energy reduction and the inspection exports.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

__device__ __forceinline__ int species_of_Z(int z) {
  switch (z) {
    case 1: return 0;
    case 6: return 1;
    case 7: return 2;
    case 8: return 3;
    case 9: return 4;
    case 16: return 5;
    case 17: return 6;
    default: return -1;
  }
}

// Element index of each atom and per-molecule element counts (create time).
__global__ void k_species_count(const int* __restrict__ Z, const int* __restrict__ mol_off,
                                int* __restrict__ species, int* __restrict__ mol_count,
                                unsigned* __restrict__ bad) {
  __shared__ int cnt[kSpecies];
  const int m = blockIdx.x;
  if (threadIdx.x < kSpecies) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int a0 = mol_off[m], a1 = mol_off[m + 1];
  for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
    const int s = species_of_Z(Z[a]);
    species[a] = s;
    if (s < 0) atomicOr(bad, 1u);
    else atomicAdd(&cnt[s], 1);
  }
  __syncthreads();
  if (threadIdx.x < kSpecies) mol_count[m * kSpecies + threadIdx.x] = cnt[threadIdx.x];
}

// Stable placement: one warp per molecule walks its atoms in caller order and
// gives each atom its internal index (molecule-contiguous, element-sorted) and
// its row (element-major).
__global__ void k_species_place(const int* __restrict__ species, const int* __restrict__ mol_off,
                                int n_mols, const int* __restrict__ mol_species_prefix,
                                const int* __restrict__ elem_mol_prefix,
                                const int* __restrict__ elem_row0, int* __restrict__ orig_of_int,
                                int* __restrict__ row_of_int, int* __restrict__ species_int,
                                int* __restrict__ mol_start, int* __restrict__ mol_end,
                                int* __restrict__ row_elem) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_mols) return;
  const int m = warp;
  const int a0 = mol_off[m], a1 = mol_off[m + 1];
  int seen[kSpecies];
#pragma unroll
  for (int s = 0; s < kSpecies; ++s) seen[s] = 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = a0; base < a1; base += 32) {
    const int a = base + lane;
    const int s = a < a1 ? species[a] : -1;
    int rank = 0;
#pragma unroll
    for (int t = 0; t < kSpecies; ++t) {
      const unsigned mask = __ballot_sync(0xffffffffu, s == t);
      if (s == t) rank = seen[t] + __popc(mask & lt);
      seen[t] += __popc(mask);
    }
    if (a < a1) {
      const int q = a0 + mol_species_prefix[m * kSpecies + s] + rank;
      const int row = elem_row0[s] + elem_mol_prefix[s * n_mols + m] + rank;
      orig_of_int[q] = a;
      row_of_int[q] = row;
      species_int[q] = s;
      mol_start[q] = a0;
      mol_end[q] = a1;
      row_elem[row] = s;
    }
  }
}

// Caller-order positions into internal order (float4), with a status bit for
// non-finite input; when forces follow, also zeroes the forces (caller order,
// FP64) and the reverse pass's overflow count.
__global__ void k_gather_positions(const float* __restrict__ pos, const int* __restrict__ orig,
                                   const int* __restrict__ species, float4* __restrict__ out, int n,
                                   unsigned* __restrict__ status, double* __restrict__ F,
                                   int* __restrict__ ovf) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0 && ovf) *ovf = 0;
  if (q >= n) return;
  const int a = orig[q];
  if (F) {
    F[3 * (size_t)a] = 0.0;
    F[3 * (size_t)a + 1] = 0.0;
    F[3 * (size_t)a + 2] = 0.0;
  }
  const float x = pos[3 * (size_t)a], y = pos[3 * (size_t)a + 1], z = pos[3 * (size_t)a + 2];
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(status, kStatNonFinite);
  out[q] = make_float4(x, y, z, __int_as_float(species[q]));  // the featurizers read the element here
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// Output layer of every network: from the third layer's pre-activation z3
// (FP32, bias included), h3 = celu(z3), y = w4 . h3 + b4, and the start of
// the reverse pass delta3 = (1/M) w4 * celu'(z3) in the products' element
// type.  One warp per (row, model).
struct ElemWidths {
  int h3[kSpecies];
};

template <typename T>
__global__ void k_head(const float* __restrict__ z3, long ldz, const int* __restrict__ row_elem,
                       const float* __restrict__ w4, const float* __restrict__ b4,
                       T* __restrict__ d3, float* __restrict__ y, int n_rows, int n_models,
                       float inv_m, ElemWidths wid) {
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long)n_rows * n_models) return;
  const int row = (int)(warp / n_models), m = (int)(warp % n_models);
  const int e = row_elem[row];
  if (e < 0) {  // padding row
    if (lane == 0) y[(size_t)row * n_models + m] = 0.f;
    return;
  }
  const int h3 = wid.h3[e];
  const float* zr = z3 + (size_t)row * ldz + (size_t)m * h3;
  T* dr = d3 + (size_t)row * ldz + (size_t)m * h3;
  const float* w = w4 + ((size_t)e * kMaxModels + m) * kH3Max;
  float acc = 0.f;
  for (int c = lane; c < h3; c += 32) {
    const float z = zr[c];
    const float ex = expf(fminf(z, 0.f) * 10.f);  // exp(z / alpha), alpha = 0.1
    const float h = z > 0.f ? z : 0.1f * expm1f(fminf(z, 0.f) * 10.f);  // no cancellation near 0
    const float dh = z > 0.f ? 1.f : ex;
    acc = fmaf(w[c], h, acc);
    dr[c] = from_f<T>(w[c] * dh * inv_m);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[(size_t)row * n_models + m] = acc + b4[e * kMaxModels + m];
}

// E_mol = sum over the molecule's atoms of (1/M) sum_m y_m, FP64.  One CTA
// per molecule, fixed reduction order (deterministic); also stores the
// per-atom ensemble means.
constexpr int kEnergyThreads = 128;
__global__ void __launch_bounds__(kEnergyThreads)
    k_energy(const float* __restrict__ y, int n_models, const int* __restrict__ row_of_int,
             const int* __restrict__ mol_off, int n_mols, double* __restrict__ E,
             double* __restrict__ atom_e) {
  __shared__ double part[kEnergyThreads / 32];
  const int m = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a0 = mol_off[m], a1 = mol_off[m + 1];
  double sum = 0.0;
  for (int q = a0 + threadIdx.x; q < a1; q += kEnergyThreads) {
    const int row = row_of_int[q];
    double e = 0.0;
    for (int k = 0; k < n_models; ++k) e += (double)y[(size_t)row * n_models + k];
    e /= n_models;
    if (atom_e) atom_e[row] = e;
    sum += e;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) part[warp] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kEnergyThreads / 32; ++w) t += part[w];
    E[m] = t;
  }
}

__global__ void k_export_neighbors(const int* __restrict__ cnt, const int* __restrict__ nbr, int cap,
                                   const int* __restrict__ orig, int n, int* __restrict__ counts_out,
                                   int* __restrict__ lists_out, int cap_out) {
  const int q = blockIdx.x;
  if (q >= n) return;
  const int a = orig[q];
  const int c = cnt[q] < cap ? cnt[q] : cap;
  if (threadIdx.x == 0) counts_out[a] = cnt[q];
  for (int t = threadIdx.x; t < cap_out; t += blockDim.x)
    lists_out[(size_t)a * cap_out + t] = t < c ? orig[nbr[(size_t)q * cap + t]] : -1;
}

template <typename T>
__global__ void k_export_features(const T* __restrict__ aev, const int* __restrict__ row_of_int,
                                  const int* __restrict__ orig, int n, int nfeat, int kpad,
                                  float* __restrict__ out, int split) {
  const int q = blockIdx.x;
  if (q >= n) return;
  const T* src = aev + (size_t)row_of_int[q] * (split ? 2 : 1) * kpad;
  float* dst = out + (size_t)orig[q] * nfeat;
  for (int f = threadIdx.x; f < nfeat; f += blockDim.x)
    dst[f] = split ? to_f(src[f]) + to_f(src[kpad + f]) : to_f(src[f]);
}

__global__ void k_export_atomic(const double* __restrict__ e_row, const int* __restrict__ row_of_int,
                                const int* __restrict__ orig, int n, double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[orig[q]] = e_row[row_of_int[q]];
}

}  // namespace

void launch_species_setup(const int* Z, const int* mol_off, int n_mols, int /*n_atoms*/,
                          int* species, int* mol_count, unsigned* bad, cudaStream_t s) {
  if (n_mols > 0) k_species_count<<<n_mols, 128, 0, s>>>(Z, mol_off, species, mol_count, bad);
}

void launch_species_place(const int* species, const int* mol_off, int n_mols,
                          const int* mol_species_prefix, const int* elem_mol_prefix,
                          const int* elem_row0, int* orig_of_int, int* row_of_int,
                          int* species_int, int* mol_start, int* mol_end, int* row_elem,
                          cudaStream_t s) {
  if (n_mols <= 0) return;
  const int threads = 128, blocks = (n_mols * 32 + threads - 1) / threads;
  k_species_place<<<blocks, threads, 0, s>>>(species, mol_off, n_mols, mol_species_prefix,
                                             elem_mol_prefix, elem_row0, orig_of_int, row_of_int,
                                             species_int, mol_start, mol_end, row_elem);
}

void launch_gather_positions(const float* pos, const int* orig, const int* species, float4* out, int n,
                             unsigned* status, double* F_zero, int* ovf_zero, cudaStream_t s) {
  if (n > 0)
    k_gather_positions<<<(n + 255) / 256, 256, 0, s>>>(pos, orig, species, out, n, status, F_zero,
                                                       ovf_zero);
}

void launch_head(const float* z3, long ldz, Prec prec, const int* row_elem, const float* w4,
                 const float* b4, void* d3, float* y, int n_rows, int n_models, const int h3[kSpecies],
                 cudaStream_t s) {
  const long warps = (long)n_rows * n_models;
  if (warps == 0) return;
  const int threads = 256;
  const long blocks = (warps * 32 + threads - 1) / threads;
  const float inv_m = 1.0f / (float)n_models;
  ElemWidths wid;
  for (int e = 0; e < kSpecies; ++e) wid.h3[e] = h3[e];
  switch (prec) {
    case Prec::F32:
      k_head<float><<<blocks, threads, 0, s>>>(z3, ldz, row_elem, w4, b4, (float*)d3, y, n_rows,
                                               n_models, inv_m, wid);
      break;
    case Prec::BF16:
      k_head<__nv_bfloat16><<<blocks, threads, 0, s>>>(z3, ldz, row_elem, w4, b4,
                                                       (__nv_bfloat16*)d3, y, n_rows, n_models,
                                                       inv_m, wid);
      break;
    case Prec::F16:
      k_head<__half><<<blocks, threads, 0, s>>>(z3, ldz, row_elem, w4, b4, (__half*)d3, y, n_rows,
                                                n_models, inv_m, wid);
      break;
  }
}

void launch_energy(const float* y, int n_models, const int* row_of_int, const int* mol_off,
                   int n_mols, double* E, double* atom_e, cudaStream_t s) {
  if (n_mols <= 0) return;
  k_energy<<<n_mols, kEnergyThreads, 0, s>>>(y, n_models, row_of_int, mol_off, n_mols, E, atom_e);
}

void launch_export_neighbors(const NeighborLists& nl, int kind, const int* orig, int n,
                             int* counts_out, int* lists_out, int cap_out, cudaStream_t s) {
  if (n <= 0) return;
  if (kind == 0)
    k_export_neighbors<<<n, 128, 0, s>>>(nl.cnt_r, nl.nbr_r, nl.cap_r, orig, n, counts_out,
                                         lists_out, cap_out);
  else
    k_export_neighbors<<<n, 128, 0, s>>>(nl.cnt_a, nl.nbr_a, nl.cap_a, orig, n, counts_out,
                                         lists_out, cap_out);
}

void launch_export_features(const void* aev, Prec prec, const int* row_of_int, const int* orig,
                            int n, int nfeat, int kpad, float* out, cudaStream_t s, bool split) {
  if (n <= 0) return;
  const int sp = split ? 1 : 0;
  switch (prec) {
    case Prec::F32:
      k_export_features<float><<<n, 256, 0, s>>>((const float*)aev, row_of_int, orig, n, nfeat, kpad, out, 0);
      break;
    case Prec::BF16:
      k_export_features<__nv_bfloat16><<<n, 256, 0, s>>>((const __nv_bfloat16*)aev, row_of_int, orig, n,
                                                         nfeat, kpad, out, sp);
      break;
    case Prec::F16:
      k_export_features<__half><<<n, 256, 0, s>>>((const __half*)aev, row_of_int, orig, n, nfeat, kpad,
                                                  out, sp);
      break;
  }
}

void launch_export_atomic_energies(const double* e_row, const int* row_of_int, const int* orig,
                                   int n, double* out, cudaStream_t s) {
  if (n > 0) k_export_atomic<<<(n + 255) / 256, 256, 0, s>>>(e_row, row_of_int, orig, n, out);
}

}  // namespace nnp
