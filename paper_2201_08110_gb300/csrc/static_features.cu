// static_features.cu -- nnp_features_static: the featurizer of one small
// molecule without any device allocation.
//
// Some callers cannot let a library allocate device memory: an MD engine that
// captures its whole time step into a CUDA graph (cudaMalloc cannot be
// captured and synchronises the device), or a host framework that hands out
// the device memory budget itself and forbids raw cudaMalloc.  For them this
// entry point computes the features of one non-periodic molecule of at most
// NNP_STATIC_MAX_ATOMS atoms with the library's own neighbour and featurizer
// kernels, keeping every intermediate (positions, neighbour lists, padded
// feature rows) in one fixed scratch array in device global memory, declared
// at file scope below.  The array is part of the library image: every GPU that
// loads the library holds it (about 1.6 MB) until the process exits.
//
// The caller passes the inputs and the output buffer.  All calls on a device
// share the one scratch array and it keeps the last call's contents, so calls
// that overlap on the GPU (different streams, different host threads) race and
// must be serialised by the caller.
#include <mutex>

#include "../../include/nnp.h"
#include "nnp_internal.cuh"

namespace nnp {

namespace {

constexpr int kStaticMax = NNP_STATIC_MAX_ATOMS;
constexpr int kStaticCap = kStaticMax;  // every other atom of the molecule fits in a list
constexpr int kStaticWarps = 4;
constexpr int kMaxDevices = 64;

struct StaticScratch {
  float4 pos[kStaticMax];
  int species[kStaticMax];
  int mol_start[kStaticMax];
  int mol_end[kStaticMax];
  int row[kStaticMax];
  int cnt_r[kStaticMax];
  int cnt_a[kStaticMax];
  int nbr_r[kStaticMax * kStaticCap];
  int nbr_a[kStaticMax * kStaticCap];
  float aev[kStaticMax * kFeaturesPad];
  unsigned bad_input;     // an atomic number outside the set, or a non-finite position
  unsigned list_status;   // neighbour-list flags (cannot overflow at this capacity)
};

// The scratch array.  In host code this name is only a stand-in for the device
// object: its address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) StaticScratch g_static_scratch;

__device__ __forceinline__ int element_index(int z) {
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

// Caller's molecule into the scratch layout: one block, one thread per atom.
// Atoms are placed in element order (stable), which the featurizer requires
// of its neighbour lists; row[] maps each placed atom back to its caller row.
__global__ void k_static_prepare(const int* __restrict__ Z, const float* __restrict__ pos, int n,
                                 StaticScratch* __restrict__ s) {
  __shared__ int elem[kStaticMax];
  const int i = threadIdx.x;
  int e = 0;
  float x = 0.f, y = 0.f, z = 0.f;
  if (i < n) {
    e = element_index(Z[i]);
    x = pos[3 * i];
    y = pos[3 * i + 1];
    z = pos[3 * i + 2];
    if (e < 0 || !(isfinite(x) && isfinite(y) && isfinite(z))) {
      atomicOr(&s->bad_input, 1u);
      e = e < 0 ? 0 : e;  // keeps every index in range; the output is poisoned below
    }
    elem[i] = e;
  }
  __syncthreads();
  if (i >= n) return;
  int slot = 0;
  for (int j = 0; j < n; ++j) {
    const int ej = elem[j];
    slot += (ej < e) || (ej == e && j < i);
  }
  s->pos[slot] = make_float4(x, y, z, __int_as_float(e));  // w: the element index, as the featurizer reads it
  s->species[slot] = e;
  s->mol_start[slot] = 0;
  s->mol_end[slot] = n;
  s->row[slot] = i;
}

__global__ void k_static_export(const StaticScratch* __restrict__ s, int n, float* __restrict__ out) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const bool bad = s->bad_input != 0u;
  const float* src = s->aev + (size_t)i * kFeaturesPad;
  for (int f = threadIdx.x; f < kFeatures; f += blockDim.x)
    out[(size_t)i * kFeatures + f] = bad ? __int_as_float(0x7fc00000) : src[f];
}

std::mutex g_setup_mutex;
StaticScratch* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

}  // namespace nnp

using namespace nnp;

extern "C" nnp_status nnp_features_static(const int32_t* Z_dev, const float* positions_dev,
                                          int32_t n_atoms, float* features_out_dev, void* stream) {
  if (n_atoms < 0) return NNP_ERR_ARG;
  if (n_atoms > kStaticMax) return NNP_ERR_TOO_LARGE;
  if (n_atoms > 0 && (!Z_dev || !positions_dev || !features_out_dev)) return NNP_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NNP_ERR_CUDA;
  if (stream) {  // the scratch address below is the current device's: so must the stream be
    int sdev = -1;
    if (cudaStreamGetDevice(static_cast<cudaStream_t>(stream), &sdev) != cudaSuccess) return NNP_ERR_ARG;
    if (sdev != dev) return NNP_ERR_ARG;
  }
  StaticScratch* p = nullptr;
  {
    // First call on this device: look up the scratch array's device address
    // (with this device current) and raise the featurizer's shared-memory limit.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) return NNP_ERR_CUDA;
      if (aev_set_smem_limits(aev_fwd_smem_bytes(kStaticCap, kStaticCap, kStaticWarps), 0) != cudaSuccess)
        return NNP_ERR_CUDA;
      g_scratch_addr[dev] = static_cast<StaticScratch*>(addr);
    }
    p = g_scratch_addr[dev];
  }
  if (n_atoms == 0) return NNP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the flags start at zero on every call; everything else is fully rewritten
  if (cudaMemsetAsync(&p->bad_input, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return NNP_ERR_CUDA;
  k_static_prepare<<<1, kStaticMax, 0, s>>>(Z_dev, positions_dev, n_atoms, p);
  AevConst c;
  const double no_box[3] = {0.0, 0.0, 0.0};
  aev_constants(c, no_box);
  Geometry g;
  g.pos = p->pos;
  g.mol_start = p->mol_start;
  g.mol_end = p->mol_end;
  g.species = p->species;
  g.n_atoms = n_atoms;
  NeighborLists nl;
  nl.cnt_r = p->cnt_r;
  nl.nbr_r = p->nbr_r;
  nl.cnt_a = p->cnt_a;
  nl.nbr_a = p->nbr_a;
  nl.cap_r = kStaticCap;
  nl.cap_a = kStaticCap;
  launch_neighbors(g, nl, c, &p->list_status, s);
  launch_aev(g, nl, c, p->row, p->aev, Prec::F32, kStaticWarps, s);
  k_static_export<<<n_atoms, 256, 0, s>>>(p, n_atoms, features_out_dev);
  return cudaGetLastError() == cudaSuccess ? NNP_OK : NNP_ERR_CUDA;
}
