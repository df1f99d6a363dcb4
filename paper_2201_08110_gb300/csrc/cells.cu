// cells.cu -- cell-list neighbour search for one large periodic region.
//
// The box is cut into n_x x n_y x n_z cells of edge >= Rcr (n = floor(L / Rcr)
// >= 2, the box being larger than twice the cutoff).  Every step the atoms are
// binned (count, scan, fill), then one warp per centre atom scans the atoms
// of its cell and the neighbouring cells (27, or fewer distinct cells when a
// dimension has fewer than 3), with the same distance test as the brute-force
// search: FP32 minimum-image distance, FP64 recheck inside the guard band.
// Accepted atoms set bits in two per-warp bitmasks over the region (radial
// and angular cutoffs); compacting the masks word by word writes every list
// in ascending internal index, i.e. grouped by element as the featurizer
// requires, and makes the result independent of the order within cells.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

__device__ __forceinline__ float3 min_image_c(float3 d, const AevConst& c) {
  d.x -= c.box[0] * rintf(d.x / c.box[0]);
  d.y -= c.box[1] * rintf(d.y / c.box[1]);
  d.z -= c.box[2] * rintf(d.z / c.box[2]);
  return d;
}

// Exact FP64 squared minimum-image distance (no contraction), as in the
// brute-force search.
__device__ double exact_d2_c(float4 xi, float4 xj, const AevConst& c) {
  double d[3] = {__dsub_rn((double)xj.x, (double)xi.x), __dsub_rn((double)xj.y, (double)xi.y),
                 __dsub_rn((double)xj.z, (double)xi.z)};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double L = c.boxd[k];
    const double n = floor(__dadd_rn(__ddiv_rn(d[k], L), 0.5));
    d[k] = __dsub_rn(d[k], __dmul_rn(L, n));
  }
  double s = __dmul_rn(d[0], d[0]);
  s = __dadd_rn(s, __dmul_rn(d[1], d[1]));
  s = __dadd_rn(s, __dmul_rn(d[2], d[2]));
  return s;
}

__device__ __forceinline__ int cell_coord(float x, float L, int n) {
  float w = x - L * floorf(x / L);  // wrap into [0, L)
  int i = (int)(w * (float)n / L);
  return min(max(i, 0), n - 1);
}

__global__ void k_cell_count(const float4* __restrict__ pos, int n, CellGrid cg, const AevConst c,
                             int* __restrict__ cell_of, int* __restrict__ count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float4 x = pos[q];
  const int ix = cell_coord(x.x, c.box[0], cg.n[0]), iy = cell_coord(x.y, c.box[1], cg.n[1]),
            iz = cell_coord(x.z, c.box[2], cg.n[2]);
  const int cell = (ix * cg.n[1] + iy) * cg.n[2] + iz;
  cell_of[q] = cell;
  atomicAdd(&count[cell], 1);
}

// Exclusive scan of the cell counts, one block.
__global__ void k_cell_scan(const int* __restrict__ count, int ncell, int* __restrict__ start) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < ncell; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < ncell ? count[i] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int ws = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < nw) warp_sums[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    const int before = carry + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (i < ncell) start[i] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void k_cell_fill(const int* __restrict__ cell_of, int n, const int* __restrict__ start,
                            int* __restrict__ fill, int* __restrict__ atoms) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int cell = cell_of[q];
  atoms[start[cell] + atomicAdd(&fill[cell], 1)] = q;
}

// Distinct neighbour-cell offsets along one dimension with n cells.
__device__ __forceinline__ int cell_offsets(int n, int (&off)[3]) {
  if (n >= 3) {
    off[0] = -1; off[1] = 0; off[2] = 1;
    return 3;
  }
  off[0] = 0; off[1] = 1;
  return n;  // n == 2: {0, 1}; n == 1: {0}
}

// Writes the set bits of a per-warp mask (words over the region) as ascending
// atom indices; returns the number of set bits (the list may be truncated at
// cap).
__device__ int compact_mask(const unsigned* mask, int words, int a0, int* out, int cap, int lane) {
  int total = 0;
  for (int base = 0; base < words; base += 32) {
    const int w = base + lane;
    unsigned bits = w < words ? mask[w] : 0u;
    const int cnt = __popc(bits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int p = total + incl - cnt;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      if (p < cap) out[p] = a0 + w * 32 + b;
      ++p;
    }
    total += __shfl_sync(0xffffffffu, incl, 31);
  }
  return total;
}

__global__ void k_neighbors_cells(Geometry g, NeighborLists nl, AevConst c, CellGrid cg,
                                  const int* __restrict__ cell_of, const int* __restrict__ start,
                                  const int* __restrict__ atoms, int words, unsigned* status) {
  extern __shared__ unsigned masks[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + warp;
  if (q >= g.n_atoms) return;  // warp-uniform
  unsigned* mR = masks + (size_t)warp * 2 * words;
  unsigned* mA = mR + words;
  for (int w = lane; w < 2 * words; w += 32) mR[w] = 0u;
  __syncwarp();
  const int a0 = g.mol_start[q];
  const float4 xi = g.pos[q];
  const int cell = cell_of[q];
  const int cz = cell % cg.n[2], cy = (cell / cg.n[2]) % cg.n[1], cx = cell / (cg.n[2] * cg.n[1]);
  int ox[3], oy[3], oz[3];
  const int nx = cell_offsets(cg.n[0], ox), ny = cell_offsets(cg.n[1], oy), nz = cell_offsets(cg.n[2], oz);
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < ny; ++b)
      for (int d = 0; d < nz; ++d) {
        const int ix = (cx + ox[a] + cg.n[0]) % cg.n[0], iy = (cy + oy[b] + cg.n[1]) % cg.n[1],
                  iz = (cz + oz[d] + cg.n[2]) % cg.n[2];
        const int cc = (ix * cg.n[1] + iy) * cg.n[2] + iz;
        for (int t = start[cc] + lane; t < start[cc + 1]; t += 32) {
          const int j = atoms[t];
          if (j == q) continue;
          const float4 xj = g.pos[j];
          const float3 dv = min_image_c(make_float3(xj.x - xi.x, xj.y - xi.y, xj.z - xi.z), c);
          const float d2 = dv.x * dv.x + dv.y * dv.y + dv.z * dv.z;
          bool inR = d2 < c.Rcr2, inA = d2 < c.Rca2;
          if (fabsf(d2 - c.Rcr2) <= 1e-4f * c.Rcr2) inR = exact_d2_c(xi, xj, c) < c.Rcr2d;
          if (fabsf(d2 - c.Rca2) <= 1e-4f * c.Rca2) inA = exact_d2_c(xi, xj, c) < c.Rca2d;
          inA = inA && inR;
          const int local = j - a0;
          if (inR) atomicOr(&mR[local >> 5], 1u << (local & 31));
          if (inA) atomicOr(&mA[local >> 5], 1u << (local & 31));
        }
      }
  __syncwarp();
  const int nr = compact_mask(mR, words, a0, nl.nbr_r + (size_t)q * nl.cap_r, nl.cap_r, lane);
  const int na = compact_mask(mA, words, a0, nl.nbr_a + (size_t)q * nl.cap_a, nl.cap_a, lane);
  if (lane == 0) {
    nl.cnt_r[q] = nr;
    nl.cnt_a[q] = na;
    if (nr > nl.cap_r) atomicOr(status, kStatCapRadial);
    if (na > nl.cap_a) atomicOr(status, kStatCapAngular);
  }
}

constexpr int kCellWarps = 4;

}  // namespace

bool cell_grid(const AevConst& c, int region_atoms, CellGrid& cg) {
  if (!c.periodic || region_atoms > kCellMaxAtoms) return false;
  for (int k = 0; k < 3; ++k) {
    // cell edge strictly above the cutoff, so rounding in the binning can
    // never put two atoms closer than the cutoff two cells apart
    cg.n[k] = (int)(c.boxd[k] / ((double)c.Rcr * 1.0001));
    if (cg.n[k] < 1) return false;
  }
  return true;
}

size_t cell_smem_bytes(int region_atoms) {
  const int words = (region_atoms + 31) / 32;
  return (size_t)kCellWarps * 2 * words * sizeof(unsigned);
}

cudaError_t cell_set_smem(size_t bytes) {
  static size_t cur = 0;
  if (bytes <= cur) return cudaSuccess;
  cur = bytes;
  return cudaFuncSetAttribute(k_neighbors_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_neighbors_cells(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                            const CellGrid& cg, const CellBuffers& cb, int region_atoms,
                            unsigned* status, cudaStream_t s) {
  const int n = g.n_atoms;
  if (n <= 0) return;
  const int ncell = cg.n[0] * cg.n[1] * cg.n[2];
  cudaMemsetAsync(cb.count, 0, sizeof(int) * ncell, s);
  cudaMemsetAsync(cb.fill, 0, sizeof(int) * ncell, s);
  k_cell_count<<<(n + 255) / 256, 256, 0, s>>>(g.pos, n, cg, c, cb.cell_of, cb.count);
  k_cell_scan<<<1, 1024, 0, s>>>(cb.count, ncell, cb.start);
  k_cell_fill<<<(n + 255) / 256, 256, 0, s>>>(cb.cell_of, n, cb.start, cb.fill, cb.atoms);
  const int words = (region_atoms + 31) / 32;
  k_neighbors_cells<<<(n + kCellWarps - 1) / kCellWarps, 32 * kCellWarps, cell_smem_bytes(region_atoms),
                      s>>>(g, nl, c, cg, cb.cell_of, cb.start, cb.atoms, words, status);
}

}  // namespace nnp
