// nnp_api.cu -- the C ABI of include/nnp.h: handle set-up (element sort,
// weight packing, work lists, buffers), the step schedule (direct launches or
// one CUDA graph replay) and the inspection exports.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nnp.h"
#include "nnp_internal.cuh"

namespace nnp {
void launch_gemm_tc(const GemmProblem* probs, const GemmTile* tiles, const int* cta_off, int n_ctas,
                    Prec p, int b_box_rows, const void* maps, unsigned* status, const int* abort_req,
                    cudaStream_t s);
void launch_gemm_tc2(const GemmProblem* probs, const GemmTile* tiles, const int* pair_off, int n_pairs,
                     Prec p, int b_half_rows, const void* maps, unsigned* status, const int* abort_req,
                     cudaStream_t s);
int tc2_max_pairs(int sms);
bool tc_available();
size_t tc_maps_bytes();
// box_cols x box_rows boxes of a [rows][cols] 16-bit matrix; 128-byte swizzle
// (64-column boxes), or 64-byte swizzle for 32-column boxes
bool tc_make_map(void* out_map, const void* base, Prec p, uint64_t rows, uint64_t cols,
                 uint64_t row_stride_elems, uint32_t box_rows, uint32_t box_cols = 64,
                 bool swizzle64 = false);
cudaError_t tc_set_smem();
}  // namespace nnp

using namespace nnp;

namespace {

thread_local std::string g_create_error;

struct Layer {
  std::vector<GemmProblem> probs;
  std::vector<GemmTile> tiles;
  std::vector<int> cta_off;  // tensor-core path: CTA c runs tiles cta_off[c] .. cta_off[c + 1]
  GemmProblem* d_probs = nullptr;
  GemmTile* d_tiles = nullptr;
  int* d_cta_off = nullptr;
};

// Longest-processing-time assignment of tiles to ctas persistent CTAs: tiles
// in decreasing cost go to the least-loaded CTA; the list is then reordered
// so that each CTA's tiles are contiguous (largest first), CTA c owning
// off[c] .. off[c + 1].  Fewer CTAs than ctas when there are fewer tiles.
void balance_tiles(std::vector<GemmTile>& tiles, const std::vector<double>& cost, int ctas,
                   std::vector<int>& off) {
  const int n = (int)tiles.size();
  ctas = std::max(1, std::min(ctas, n));
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(ctas, 0.0);
  std::vector<std::vector<int>> own(ctas);
  for (int i : order) {
    int best = 0;
    for (int c = 1; c < ctas; ++c)
      if (load[c] < load[best]) best = c;
    load[best] += cost[i];
    own[best].push_back(i);
  }
  std::vector<GemmTile> out;
  out.reserve(n);
  off.assign(1, 0);
  for (int c = 0; c < ctas; ++c) {
    for (int i : own[c]) out.push_back(tiles[i]);
    off.push_back((int)out.size());
  }
  tiles.swap(out);
}

size_t elem_size(Prec p) { return p == Prec::F32 ? 4 : 2; }


}  // namespace

struct nnp_ctx {
  int dev = 0;
  int n_atoms = 0, n_mols = 0, n_models = 1;
  Prec prec = Prec::F32;
  int use_graph = 0;
  int split = 0;           // 16-bit networks: forward products on split (hi, lo) operands
  int aev_aliased = 0;     // the features share their buffer with dE/dG
  bool features_overwritten = false;  // the last step's reverse pass wrote over the features
  int test_abort = 0;
  int single_cta = 0;  // the first layer on single CTAs even where pairs fit
  ModelDesc md{};  // the model: elements, feature layout, network widths
  AevConst aevc{};
  int elem_count[kSpecies] = {0};
  int elem_row0[kSpecies + 1] = {0};
  int n_rows = 0;
  int max_mol = 0;
  long ldh1 = 0, ldh2 = 0, ldz3 = 0;

  // device: layout
  int *d_Z = nullptr, *d_mol_off = nullptr, *d_orig = nullptr, *d_row_of_int = nullptr,
      *d_species_int = nullptr, *d_mol_start = nullptr, *d_mol_end = nullptr, *d_row_elem = nullptr;
  float4* d_pos = nullptr;
  NeighborLists nl{};
  // device: activations
  void *d_aev = nullptr, *d_h1 = nullptr, *d_h2 = nullptr, *d_d3 = nullptr;
  float* d_z3 = nullptr;  // third-layer pre-activation, FP32 (not a product operand)
  float *d_y = nullptr, *d_dG = nullptr;
  double* d_atom_e = nullptr;
  unsigned* d_status = nullptr;
  int* d_abort = nullptr;  // tests: nonzero makes the tensor-core kernels abort at their start
  int abort_steps = 0;     // tests: evaluations left that start with d_abort set
  // device: weights
  void* d_w = nullptr;
  float* d_b = nullptr;
  float *d_w4 = nullptr, *d_b4 = nullptr;
  size_t w_off[6] = {0};  // W1, W2, W3, W3T, W2T, W1T element offsets in d_w
  Layer L[6];              // 0 L1 fwd, 1 L2 fwd, 2 L3 fwd, 3 L3 rev, 4 L2 rev, 5 L1 rev
  void* d_maps = nullptr;
  bool use_cells = false;
  CellGrid cells{};
  CellBuffers cellbuf{};
  alignas(64) unsigned char tc_maps[6][384];  // tensor-core path: {A, B, D} TMA descriptors per layer
  alignas(64) unsigned char tail_maps[6 * 128];  // fused tail: h1, w2, w3, w3t, w2t, h1 (32-col boxes)
  std::vector<TailProblem> tail_probs;
  std::vector<GemmTile> tail_tiles;
  std::vector<int> tail_off;  // CTA c runs tail tiles tail_off[c] .. tail_off[c + 1]
  int* d_tail_off = nullptr;
  int sms = 152;
  TailProblem* d_tail_probs = nullptr;
  GemmTile* d_tail_tiles = nullptr;
  // reverse pass work list
  int4* d_work = nullptr;
  int* d_ovf = nullptr;  // reverse pass: [0] count, [1..] deferred centres
  int4* d_nbr_work = nullptr;  // neighbour search: chunks of centres of one molecule
  int n_nbr_work = 0;
  int n_work = 0;
  int fwd_warps = 4, adj_warps = 4, adj_chunk = 0, adj_shared_acc = 1, smem_atoms_max = 0;
  int adj_ovf_ctas = 304;  // CTAs of the reverse pass's overflow launch
  int l1_bn = 256;                  // N tile of the first layer's products (tensor cores)
  bool l1_pairs = true;             // the first layer's products on CTA pairs (256-row tiles)
  int l1_max_pairs = 0;             // CTA pairs that fit on the GPU at once
  int tc_box[6] = {256, kH2Max, kH3Max, kH2Max, kH1Max, 256};  // weight-box rows per layer
  std::vector<int> mol_off_h;
  const void* l1_b_base[2] = {nullptr, nullptr};  // W1, W1T (tensor-core maps of layers 0, 5)
  uint64_t l1_b_rows[2] = {0, 0}, l1_b_cols[2] = {0, 0};
  // host-buffer entry point
  float* d_pos_in = nullptr;
  double *d_E = nullptr, *d_F = nullptr;
  // graph
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side = nullptr;  // the energy reduction runs beside the reverse pass
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const float* g_pos = nullptr;
  double *g_E = nullptr, *g_F = nullptr;
  cudaStream_t last_stream = nullptr;
  std::string err;

  Geometry geometry() const {
    Geometry g;
    g.pos = d_pos;
    g.mol_start = d_mol_start;
    g.mol_end = d_mol_end;
    g.species = d_species_int;
    g.n_atoms = n_atoms;
    return g;
  }
};

namespace {

nnp_status fail(nnp_ctx* h, nnp_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

// A failed call's error is also taken off the thread's last-error state, so
// that it does not surface in a later, unrelated call.
#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      cudaGetLastError();                                                               \
      return fail(h, e_ == cudaErrorMemoryAllocation ? NNP_ERR_ALLOC : NNP_ERR_CUDA,    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    }                                                                                   \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

// ANI-2x (model 0): cutoffs 5.1 / 3.5 A, EtaR 19.7, EtaA 12.5, Zeta 14.1, shift
// grids as closed linspaces (radial 0.8 .. 4.9 A in 16, angular distance
// 0.8 .. 3.1 A in 8, angle 0.39 .. 2.75 rad in 4).  ANI-1x (model 1): 5.2 /
// 3.5 A, EtaR 16, EtaA 8, Zeta 32, radial shifts 0.9 + 0.26875 k A (16),
// angular distance shifts 0.9 + 0.65 a A (4), angle shifts pi/16 + z pi/8 (8).
// Both: the featurizer functions of Sec. 1 (ANI's modified Behler-Parrinello
// symmetry functions).
void init_aev_const(AevConst& c, const double box[3], int model) {
  std::memset(&c, 0, sizeof(c));
  const bool x1 = model == 1;
  const int ns = x1 ? 4 : kSpecies, na = x1 ? 4 : 8, nz = x1 ? 8 : 4;
  c.model = x1 ? 1 : 0;
  c.Rcr = x1 ? 5.2f : 5.1f;
  c.Rca = 3.5f;
  c.Rcr2 = c.Rcr * c.Rcr;
  c.Rca2 = c.Rca * c.Rca;
  c.Rcr2d = (double)c.Rcr * (double)c.Rcr;
  c.Rca2d = (double)c.Rca * (double)c.Rca;
  c.EtaR = x1 ? 16.f : 19.7f;
  c.EtaA = x1 ? 8.f : 12.5f;
  c.Zeta = x1 ? (float)ShapeANI1x::kZetaInt : 14.1f;  // the ANI-1x kernels raise to 32 by multiplication
  const double pi = 3.14159265358979323846;
  double shr[kShfR], sha[kMaxShfA];
  for (int k = 0; k < kShfR; ++k) shr[k] = x1 ? 0.9 + 0.26875 * k : 0.8 + (4.9 - 0.8) * k / (kShfR - 1);
  for (int k = 0; k < na; ++k) sha[k] = x1 ? 0.9 + 0.65 * k : 0.8 + (3.1 - 0.8) * k / (na - 1);
  for (int k = 0; k < kShfR; ++k) c.ShfR[k] = (float)shr[k];
  for (int k = 0; k < na; ++k) c.ShfA[k] = (float)sha[k];
  for (int k = 0; k < nz; ++k) {
    const double z = x1 ? pi / 16.0 + k * pi / 8.0 : 0.39 + (2.75 - 0.39) * k / (nz - 1);
    c.cosZ[k] = (float)std::cos(z);
    c.sinZ[k] = (float)std::sin(z);
  }
  const double log2e = 1.4426950408889634;
  const double sqR = std::sqrt((double)c.EtaR * log2e), sqA = std::sqrt((double)c.EtaA * log2e);
  auto hi = [](double v) { return (float)v; };
  auto lo = [](double v) { return (float)(v - (double)(float)v); };
  c.sqEtaR = hi(sqR);
  c.sqEtaRl = lo(sqR);
  c.sqEtaA = hi(sqA);
  c.sqEtaAl = lo(sqA);
  for (int k = 0; k < kShfR; ++k) {
    c.ShfRs[k] = hi(sqR * shr[k]);
    c.ShfRsl[k] = lo(sqR * shr[k]);
  }
  for (int k = 0; k < na; ++k) {
    c.ShfAs[k] = hi(sqA * sha[k]);
    c.ShfAsl[k] = lo(sqA * sha[k]);
  }
  c.gradR = (float)(-2.0 * (double)c.EtaR / sqR);
  c.gradA = (float)(-2.0 * (double)c.EtaA / sqA);
  c.hsqEtaA = 0.5f * c.sqEtaA;  // exact halving of the pair
  c.hsqEtaAl = 0.5f * c.sqEtaAl;
  c.hgradA = (float)(-(double)c.EtaA / sqA);
  c.dcosA = (float)(0.95 * (double)c.Zeta);
  int p = 0;
  for (int s = 0; s < ns; ++s)
    for (int t = s; t < ns; ++t) {
      c.pair_index[s][t] = p;
      c.pair_index[t][s] = p;
      ++p;
    }
  c.periodic = (box[0] != 0.0 || box[1] != 0.0 || box[2] != 0.0) ? 1 : 0;
  for (int k = 0; k < 3; ++k) {
    c.boxd[k] = box[k];
    c.box[k] = (float)box[k];
  }
}

// Parameters of one element's network in the caller's weight layout: W1
// [h1][nfeat], b1, W2 [h2][h1], b2, W3 [h3][h2], b3, w4 [h3], b4.
long element_params(const ModelDesc& md, int e) {
  const long n0 = md.nfeat, n1 = md.hidden[e][0], n2 = md.hidden[e][1], n3 = md.hidden[e][2];
  return n1 * n0 + n1 + n2 * n1 + n2 + n3 * n2 + n3 + n3 + 1;
}

long model_params(const ModelDesc& md) {
  long s = 0;
  for (int e = 0; e < md.ns; ++e) s += element_params(md, e);
  return s;
}

uint16_t f2bf(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

uint16_t f2h(float f) {  // IEEE binary16, round to nearest even
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u;
  int32_t exp = (int32_t)((x >> 23) & 0xff) - 127 + 15;
  uint32_t man = x & 0x7fffffu;
  if (((x >> 23) & 0xff) == 0xff) return (uint16_t)(sign | 0x7c00u | (man ? 0x200u : 0u));
  if (exp >= 31) return (uint16_t)(sign | 0x7c00u);
  if (exp <= 0) {
    if (exp < -10) return (uint16_t)sign;
    man |= 0x800000u;
    const int shift = 14 - exp;
    uint32_t h = man >> shift;
    const uint32_t rem = man & ((1u << shift) - 1u), half = 1u << (shift - 1);
    if (rem > half || (rem == half && (h & 1u))) ++h;
    return (uint16_t)(sign | h);
  }
  uint32_t h = ((uint32_t)exp << 10) | (man >> 13);
  const uint32_t rem = man & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;
  return (uint16_t)(sign | h);
}

float bf2f(uint16_t u) {
  const uint32_t x = (uint32_t)u << 16;
  float f;
  std::memcpy(&f, &x, 4);
  return f;
}

float h2f(uint16_t u) {  // IEEE binary16 to FP32 (exact)
  const uint32_t sign = (uint32_t)(u & 0x8000u) << 16;
  const int exp = (u >> 10) & 0x1f;
  const uint32_t man = u & 0x3ffu;
  float f;
  if (exp == 0) {  // zero or subnormal: man * 2^-24
    f = std::ldexp((float)man, -24);
    return sign ? -f : f;
  }
  const uint32_t x = exp == 31 ? (sign | 0x7f800000u | (man << 13))
                               : (sign | ((uint32_t)(exp - 15 + 127) << 23) | (man << 13));
  std::memcpy(&f, &x, 4);
  return f;
}

// Packs host FP32 values into the device element type.
struct Packer {
  Prec p;
  std::vector<float> f32;
  std::vector<uint16_t> f16;
  void resize(size_t n) {
    if (p == Prec::F32) f32.assign(n, 0.f);
    else f16.assign(n, 0);
  }
  void set(size_t i, float v) {
    if (p == Prec::F32) f32[i] = v;
    else f16[i] = p == Prec::BF16 ? f2bf(v) : f2h(v);
  }
  // a forward weight: with split, hi = round(v) at i and lo = round(v - hi)
  // lo_off elements to its right
  void set_fwd(size_t i, size_t lo_off, float v, int split) {
    set(i, v);
    if (split) set(i + lo_off, v - (p == Prec::BF16 ? bf2f(f16[i]) : h2f(f16[i])));
  }
  const void* data() const { return p == Prec::F32 ? (const void*)f32.data() : (const void*)f16.data(); }
};

void add_tiles(Layer& L, int bm, int bn) {
  const int pi = (int)L.probs.size() - 1;
  const GemmProblem& P = L.probs.back();
  for (int m0 = 0; m0 < P.M; m0 += bm)
    for (int n0 = 0; n0 < P.N; n0 += bn) L.tiles.push_back(GemmTile{pi, m0, n0, 0});
}

}  // namespace

namespace nnp {
// The featurizer constants, for other translation units of the library.
void aev_constants(AevConst& c, const double box[3], int model) { init_aev_const(c, box, model); }

// ANI-2x: H, C, N, O, F, S, Cl; widths H 256-192-160, C 224-192-160, N and O
// 192-160-128, F, S and Cl 160-128-96.  ANI-1x: H, C, N, O; widths H
// 160-128-96, C 144-112-96, N and O 128-112-96 (device widths C 160-128-96,
// N and O 128-128-96).
bool model_desc(int id, ModelDesc& md) {
  std::memset(&md, 0, sizeof(md));
  static const int z7[7] = {1, 6, 7, 8, 9, 16, 17};
  static const int h2x[7][3] = {{256, 192, 160}, {224, 192, 160}, {192, 160, 128}, {192, 160, 128},
                                {160, 128, 96},  {160, 128, 96},  {160, 128, 96}};
  static const int h1x[4][3] = {{160, 128, 96}, {144, 112, 96}, {128, 112, 96}, {128, 112, 96}};
  if (id != 0 && id != 1) return false;
  md.id = id;
  md.ns = id == 1 ? 4 : 7;
  md.na = id == 1 ? 4 : 8;
  md.nz = 32 / md.na;
  md.nfeat = id == 1 ? ShapeANI1x::kFeat : ShapeANI2x::kFeat;
  md.kpad = id == 1 ? ShapeANI1x::kPad : ShapeANI2x::kPad;
  md.Rcr = id == 1 ? 5.2f : 5.1f;
  md.Rca = 3.5f;
  for (int e = 0; e < md.ns; ++e) {
    md.z[e] = z7[e];
    for (int l = 0; l < 3; ++l) {
      md.hidden[e][l] = id == 1 ? h1x[e][l] : h2x[e][l];
      md.hpad[e][l] = (md.hidden[e][l] + 31) / 32 * 32;
    }
  }
  return true;
}
}  // namespace nnp

namespace {

// Reverse-pass work list: (molecule, chunk of centres) items, largest first,
// and the per-warp shared-memory accumulator limit for the given warps per CTA.
// shared_acc: 1 = per-warp FP64 accumulators of the molecule in shared
// memory (molecules that fit), 0 = FP64 atomics straight into the forces.
nnp_status build_work_list(nnp_ctx* h, int warps, int chunk, int shared_acc = 1) {
  const size_t budget = 160 * 1024;
  const size_t fixed = aev_adj_smem_bytes(h->nl.cap_r, aev_adj_stage_cap(h->nl.cap_a), warps, 0);
  int smax = 0;
  if (shared_acc && fixed < budget)
    smax = (int)std::min<size_t>((budget - fixed) / ((size_t)warps * 24), 1 << 20);
  smax = std::min(smax, h->max_mol);
  smax = (smax / 2) * 2;
  h->adj_shared_acc = shared_acc;
  std::vector<int4> work;
  std::vector<long> cost;
  const int n_mols = h->n_mols;
  for (int m = 0; m < n_mols; ++m) {
    const int a0 = h->mol_off_h[m], n = h->mol_off_h[m + 1] - a0;
    for (int c0 = 0; c0 < n; c0 += chunk) {
      work.push_back(make_int4(a0, n, a0 + c0, a0 + std::min(n, c0 + chunk)));
      cost.push_back((long)std::min(chunk, n - c0) * n);
    }
  }
  std::vector<int> order(work.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int4> sorted(work.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = work[order[i]];
  if (h->d_work) cudaFree(h->d_work);
  h->d_work = nullptr;
  CK(dalloc(&h->d_work, sorted.size()));
  if (!sorted.empty())
    CK(cudaMemcpy(h->d_work, sorted.data(), sizeof(int4) * sorted.size(), cudaMemcpyHostToDevice));
  h->n_work = (int)sorted.size();
  h->smem_atoms_max = smax;
  h->adj_warps = warps;
  h->adj_chunk = chunk;
  CK(aev_set_smem_limits(0, aev_adj_launch_smem(h->nl.cap_r, h->nl.cap_a, warps, smax)));
  h->adj_ovf_ctas = aev_adj_overflow_ctas(h->nl.cap_r, h->nl.cap_a, warps, h->md.id);
  return NNP_OK;
}

// Tiles (and, on tensor cores, the weight maps) of the first layer's two
// products for an N tile of bn columns.  On CTA pairs (h->l1_pairs) a tile
// has 256 rows and the units that share out the tiles are the SM pairs; each
// CTA's B box holds half the tile's columns.
nnp_status set_l1_tiles(nnp_ctx* h, int bn) {
  const int bm = h->l1_pairs ? 256 : 128;
  for (int layer : {0, 5}) {
    Layer& L = h->L[layer];
    L.tiles.clear();
    std::vector<double> cost;
    for (int pi = 0; pi < (int)L.probs.size(); ++pi) {
      const GemmProblem& P = L.probs[pi];
      for (int m0 = 0; m0 < P.M; m0 += bm)
        for (int n0 = 0; n0 < P.N; n0 += bn) {
          L.tiles.push_back(GemmTile{pi, m0, n0, 0});
          cost.push_back((double)P.K * std::min(bn, P.N - n0));
        }
    }
    // the last, partly filled wave: split its cheapest tiles into 2 or 4
    // column pieces so they spread over more CTAs.  A piece is a whole number
    // of 64-column output boxes: the epilogue stores whole boxes (zeros past
    // a tile's columns), which past a piece would land in its neighbour's
    const int S = h->l1_pairs ? h->l1_max_pairs : h->sms, r = (int)L.tiles.size() % S;
    const int k = (r > 0 && 4 * r <= S) ? 4 : (r > 0 && 2 * r <= S) ? 2 : 1;
    if (k > 1 && bn / k >= 64) {
      std::vector<int> order(L.tiles.size());
      for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] < cost[b]; });
      std::vector<GemmTile> extra;
      std::vector<double> extra_cost;
      for (int q = 0; q < r; ++q) {
        const int i = order[q];
        GemmTile& t = L.tiles[i];
        const int w = std::min(bn, L.probs[t.problem].N - t.n0);
        if (w % (64 * k)) continue;
        const int pw = w / k;
        for (int piece = 1; piece < k; ++piece) {
          extra.push_back(GemmTile{t.problem, t.m0, t.n0 + piece * pw, pw});
          extra_cost.push_back(cost[i] / k);
        }
        t.width = pw;
        cost[i] /= k;
      }
      L.tiles.insert(L.tiles.end(), extra.begin(), extra.end());
      cost.insert(cost.end(), extra_cost.begin(), extra_cost.end());
    }
    balance_tiles(L.tiles, cost, S, L.cta_off);
    if (L.d_tiles) cudaFree(L.d_tiles);
    if (L.d_cta_off) cudaFree(L.d_cta_off);
    L.d_tiles = nullptr;
    L.d_cta_off = nullptr;
    CK(dalloc(&L.d_tiles, L.tiles.size()));
    CK(dalloc(&L.d_cta_off, L.cta_off.size()));
    if (!L.tiles.empty())
      CK(cudaMemcpy(L.d_tiles, L.tiles.data(), sizeof(GemmTile) * L.tiles.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.d_cta_off, L.cta_off.data(), sizeof(int) * L.cta_off.size(), cudaMemcpyHostToDevice));
    const int i = layer == 0 ? 0 : 1;
    const int box_rows = h->l1_pairs ? bn / 2 : bn;
    if (!tc_make_map(h->tc_maps[layer] + 128, h->l1_b_base[i], h->prec, h->l1_b_rows[i],
                     h->l1_b_cols[i], h->l1_b_cols[i], (uint32_t)box_rows))
      return fail(h, NNP_ERR_CUDA, "cuTensorMapEncodeTiled failed for the first layer");
    h->tc_box[layer] = box_rows;
  }
  h->l1_bn = bn;
  return NNP_OK;
}

}  // namespace

extern "C" {

int64_t nnp_weights_per_model(void) { return nnp_weights_per_model_of(NNP_MODEL_ANI2X); }
int32_t nnp_num_features(void) { return nnp_num_features_of(NNP_MODEL_ANI2X); }

int64_t nnp_weights_per_model_of(int32_t model) {
  ModelDesc md;
  return model_desc(model, md) ? model_params(md) : -1;
}

int32_t nnp_num_features_of(int32_t model) {
  ModelDesc md;
  return model_desc(model, md) ? md.nfeat : -1;
}

const char* nnp_last_error(nnp_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void nnp_destroy(nnp_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->aev_aliased) h->d_aev = nullptr;  // the dE/dG buffer
  void* ptrs[] = {h->d_Z, h->d_mol_off, h->d_orig, h->d_row_of_int, h->d_species_int,
                  h->d_mol_start, h->d_mol_end, h->d_row_elem, h->d_pos, h->nl.cnt_r,
                  h->nl.nbr_r, h->nl.cnt_a, h->nl.nbr_a, h->d_aev, h->d_h1,
                  h->d_h2, h->d_z3, h->d_d3, h->d_y, h->d_dG, h->d_atom_e, h->d_status, h->d_abort, h->d_w, h->d_b,
                  h->d_w4, h->d_b4, h->d_maps, h->d_work, h->d_ovf, h->d_nbr_work, h->d_pos_in, h->d_E, h->d_F};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& L : h->L) {
    if (L.d_probs) cudaFree(L.d_probs);
    if (L.d_tiles) cudaFree(L.d_tiles);
    if (L.d_cta_off) cudaFree(L.d_cta_off);
  }
  if (h->d_tail_off) cudaFree(h->d_tail_off);
  for (void* p : {(void*)h->cellbuf.cell_of, (void*)h->cellbuf.count, (void*)h->cellbuf.start,
                  (void*)h->cellbuf.fill, (void*)h->cellbuf.atoms})
    if (p) cudaFree(p);
  if (h->d_tail_probs) cudaFree(h->d_tail_probs);
  if (h->d_tail_tiles) cudaFree(h->d_tail_tiles);
  delete h;
}

nnp_status nnp_create(const int32_t* Z, int32_t n_atoms, const nnp_params* params, nnp_handle* out) {
  if (n_atoms < 0) return fail(nullptr, NNP_ERR_ARG, "n_atoms < 0");
  const int32_t off[2] = {0, n_atoms};
  return nnp_create_batch(Z, off, 1, params, out);
}

nnp_status nnp_create_batch(const int32_t* Z, const int32_t* mol_offsets, int32_t n_mols,
                            const nnp_params* params, nnp_handle* out) {
  nnp_ctx* h = nullptr;
  if (!out || !params || !mol_offsets || n_mols < 0) return fail(nullptr, NNP_ERR_ARG, "null argument");
  *out = nullptr;
  if (mol_offsets[0] != 0) return fail(nullptr, NNP_ERR_ARG, "mol_offsets[0] != 0");
  for (int m = 0; m < n_mols; ++m)
    if (mol_offsets[m + 1] < mol_offsets[m]) return fail(nullptr, NNP_ERR_ARG, "mol_offsets decreasing");
  const int N = mol_offsets[n_mols];
  if (N > 0 && !Z) return fail(nullptr, NNP_ERR_ARG, "Z is null");
  if (params->total_charge != 0)
    return fail(nullptr, NNP_ERR_CHARGE, "total charge must be 0 (neutral molecules only)");
  if (params->n_models < 1 || params->n_models > kMaxModels)
    return fail(nullptr, NNP_ERR_ARG, "n_models must be in [1, 16]");
  if (params->precision < 0 || params->precision > 2) return fail(nullptr, NNP_ERR_ARG, "bad precision");
  ModelDesc md;
  if (!model_desc(params->model, md)) return fail(nullptr, NNP_ERR_ARG, "model must be 0 (ANI-2x) or 1 (ANI-1x)");
  if (!params->weights || params->n_weights != model_params(md) * params->n_models)
    return fail(nullptr, NNP_ERR_ARG, "weights: expected n_models * nnp_weights_per_model_of(model) floats");
  for (int r = 0; r < 2; ++r)
    if (params->reserved[r] != 0) return fail(nullptr, NNP_ERR_ARG, "reserved fields must be zero");
  if ((params->single_pass | params->recompute_aev | params->test_abort | params->single_cta) & ~1)
    return fail(nullptr, NNP_ERR_ARG, "single_pass, recompute_aev, test_abort and single_cta must be 0 or 1");
  if (params->neighbor_mode < 0 || params->neighbor_mode > 2)
    return fail(nullptr, NNP_ERR_ARG, "neighbor_mode must be 0, 1 or 2");
  for (int i = 0; i < N; ++i) {
    const int z = Z[i];
    bool known = false;
    for (int e = 0; e < md.ns; ++e) known = known || md.z[e] == z;
    if (!known)
      return fail(nullptr, NNP_ERR_SPECIES, "unsupported atomic number " + std::to_string(z) +
                                                 " at atom " + std::to_string(i) + " for this model");
  }
  const bool periodic = params->box[0] != 0.0 || params->box[1] != 0.0 || params->box[2] != 0.0;
  if (periodic)
    for (int k = 0; k < 3; ++k)
      if (!(params->box[k] > 2.0 * (double)md.Rcr))
        return fail(nullptr, NNP_ERR_ARG, "box edge must exceed twice the radial cutoff");
  if (params->max_neighbors < 0 || params->max_angular < 0)
    return fail(nullptr, NNP_ERR_ARG, "negative capacity");

  h = new (std::nothrow) nnp_ctx();
  if (!h) return fail(nullptr, NNP_ERR_ALLOC, "host allocation failed");
  cudaGetLastError();  // a stale error of the caller's must not be taken for one of these launches
  struct Guard {
    nnp_ctx*& h;
    bool ok = false;
    ~Guard() {
      if (!ok && h) {
        g_create_error = h->err;
        nnp_destroy(h);
      }
    }
  } guard{h};

  cudaGetDevice(&h->dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
  if (h->sms <= 0) h->sms = 152;
  h->n_atoms = N;
  h->n_mols = n_mols;
  h->n_models = params->n_models;
  h->prec = (Prec)params->precision;
  h->use_graph = params->use_graph;
  h->split = (h->prec != Prec::F32 && !params->single_pass) ? 1 : 0;
  h->aev_aliased = params->recompute_aev;
  h->test_abort = params->test_abort;
  h->single_cta = params->single_cta;
  h->md = md;
  init_aev_const(h->aevc, params->box, md.id);
  for (int m = 0; m < n_mols; ++m) h->max_mol = std::max(h->max_mol, mol_offsets[m + 1] - mol_offsets[m]);
  if (h->prec != Prec::F32 && !tc_available())
    return fail(h, NNP_ERR_UNSUPPORTED, "tensor-core path needs an sm_103a device");

  const int M = h->n_models;
  cudaStream_t s0 = nullptr;
  CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  s0 = h->cap_stream;

  // ---- element sort on the device (a1) ----
  int* d_species_caller = nullptr;
  int* d_mol_count = nullptr;
  CK(dalloc(&h->d_Z, N));
  CK(dalloc(&h->d_mol_off, n_mols + 1));
  CK(dalloc(&d_species_caller, N));
  CK(dalloc(&d_mol_count, (size_t)n_mols * kSpecies));
  CK(dalloc(&h->d_status, 1));
  CK(cudaMemset(h->d_status, 0, sizeof(unsigned)));
  CK(dalloc(&h->d_abort, 1));
  CK(cudaMemset(h->d_abort, 0, sizeof(int)));
  h->abort_steps = params->test_abort;
  if (N) CK(cudaMemcpy(h->d_Z, Z, sizeof(int) * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_mol_off, mol_offsets, sizeof(int) * (n_mols + 1), cudaMemcpyHostToDevice));
  launch_species_setup(h->d_Z, h->d_mol_off, n_mols, N, d_species_caller, d_mol_count, h->d_status, s0);
  CK(cudaGetLastError());
  std::vector<int> mol_count((size_t)n_mols * kSpecies);
  CK(cudaStreamSynchronize(s0));
  if (n_mols)
    CK(cudaMemcpy(mol_count.data(), d_mol_count, sizeof(int) * mol_count.size(), cudaMemcpyDeviceToHost));
  // prefix sums (host, create time)
  std::vector<int> mol_species_prefix((size_t)n_mols * kSpecies), elem_mol_prefix((size_t)kSpecies * n_mols);
  for (int m = 0; m < n_mols; ++m) {
    int acc = 0;
    for (int s = 0; s < kSpecies; ++s) {
      mol_species_prefix[(size_t)m * kSpecies + s] = acc;
      acc += mol_count[(size_t)m * kSpecies + s];
    }
  }
  for (int s = 0; s < kSpecies; ++s) {
    int acc = 0;
    for (int m = 0; m < n_mols; ++m) {
      elem_mol_prefix[(size_t)s * n_mols + m] = acc;
      acc += mol_count[(size_t)m * kSpecies + s];
    }
    h->elem_count[s] = acc;
  }
  h->elem_row0[0] = 0;
  for (int s = 0; s < kSpecies; ++s)
    h->elem_row0[s + 1] = h->elem_row0[s] + ((h->elem_count[s] + kRowAlign - 1) / kRowAlign) * kRowAlign;
  h->n_rows = std::max(h->elem_row0[kSpecies], kRowAlign);

  int *d_msp = nullptr, *d_emp = nullptr, *d_er0 = nullptr;
  CK(dalloc(&d_msp, mol_species_prefix.size()));
  CK(dalloc(&d_emp, elem_mol_prefix.size()));
  CK(dalloc(&d_er0, kSpecies + 1));
  if (!mol_species_prefix.empty()) {
    CK(cudaMemcpy(d_msp, mol_species_prefix.data(), sizeof(int) * mol_species_prefix.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_emp, elem_mol_prefix.data(), sizeof(int) * elem_mol_prefix.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(d_er0, h->elem_row0, sizeof(int) * (kSpecies + 1), cudaMemcpyHostToDevice));
  CK(dalloc(&h->d_orig, N));
  CK(dalloc(&h->d_ovf, N + 1));
  CK(dalloc(&h->d_row_of_int, N));
  CK(dalloc(&h->d_species_int, N));
  CK(dalloc(&h->d_mol_start, N));
  CK(dalloc(&h->d_mol_end, N));
  CK(dalloc(&h->d_row_elem, h->n_rows));
  CK(cudaMemset(h->d_row_elem, 0xff, sizeof(int) * h->n_rows));
  launch_species_place(d_species_caller, h->d_mol_off, n_mols, d_msp, d_emp, d_er0, h->d_orig,
                       h->d_row_of_int, h->d_species_int, h->d_mol_start, h->d_mol_end,
                       h->d_row_elem, s0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s0));
  cudaFree(d_species_caller);
  cudaFree(d_mol_count);
  cudaFree(d_msp);
  cudaFree(d_emp);
  cudaFree(d_er0);

  // ---- neighbour lists ----
  auto round32 = [](int x) { return ((x + 31) / 32) * 32; };
  int cap_r = params->max_neighbors;
  if (cap_r == 0) cap_r = std::min(std::max(round32(h->max_mol - 1), 32), 256);
  int cap_a = params->max_angular;
  if (cap_a == 0) cap_a = std::min(cap_r, 160);
  cap_r = round32(cap_r);
  cap_a = round32(std::min(cap_a, cap_r));
  if (cap_a > 255) cap_a = 256;
  h->nl.cap_r = cap_r;
  h->nl.cap_a = cap_a;
  {  // cell list for one large periodic region
    const int mode = params->neighbor_mode;
    const bool want = mode == 2 || (mode == 0 && n_mols == 1 && N > 1024);
    if (want && h->aevc.periodic && n_mols == 1 && cell_grid(h->aevc, N, h->cells)) {
      const int ncell = h->cells.n[0] * h->cells.n[1] * h->cells.n[2];
      CK(dalloc(&h->cellbuf.cell_of, N));
      CK(dalloc(&h->cellbuf.count, ncell));
      CK(dalloc(&h->cellbuf.start, ncell + 1));
      CK(dalloc(&h->cellbuf.fill, ncell));
      CK(dalloc(&h->cellbuf.atoms, N));
      CK(cell_set_smem(cell_smem_bytes(N)));
      h->use_cells = true;
    } else if (mode == 2) {
      return fail(h, NNP_ERR_UNSUPPORTED,
                  "cell list needs one periodic region of at most 32768 atoms");
    }
  }
  if (!h->use_cells) {  // all-pairs search per molecule: work items of nbr_chunk() centres, largest first
    std::vector<int4> work;
    std::vector<long> cost;
    for (int m = 0; m < n_mols; ++m) {
      const int a0 = mol_offsets[m], n = mol_offsets[m + 1] - a0;
      for (int c0 = 0; c0 < n; c0 += nbr_chunk()) {
        const int c1 = std::min(n, c0 + nbr_chunk());
        work.push_back(make_int4(a0, n, a0 + c0, a0 + c1));
        cost.push_back((long)(c1 - c0) * n);
      }
    }
    std::vector<int> order(work.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<int4> sorted(work.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = work[order[i]];
    h->n_nbr_work = (int)sorted.size();
    CK(dalloc(&h->d_nbr_work, sorted.size()));
    if (!sorted.empty())
      CK(cudaMemcpy(h->d_nbr_work, sorted.data(), sizeof(int4) * sorted.size(), cudaMemcpyHostToDevice));
    CK(nbr_set_smem(nbr_smem_bytes(h->max_mol)));
  }
  CK(dalloc(&h->d_pos, N));
  CK(dalloc(&h->nl.cnt_r, N));
  CK(dalloc(&h->nl.cnt_a, N));
  CK(dalloc(&h->nl.nbr_r, (size_t)N * cap_r));
  CK(dalloc(&h->nl.nbr_a, (size_t)N * cap_a));

  // ---- activations ----
  const size_t es = elem_size(h->prec);
  const int sp = h->split ? 2 : 1;  // hi and lo halves side by side
  h->ldh1 = (long)sp * M * kH1Max;
  h->ldh2 = (long)M * kH2Max;
  h->ldz3 = (long)M * kH3Max;
  const size_t R = h->n_rows;
  // dE/dG [R][kpad] FP32; with recompute_aev the features (at most as large:
  // [R][kpad] FP32 or [R][2 x kpad] 16-bit) live in the same buffer
  const size_t kpad = (size_t)md.kpad;
  CK(dalloc(&h->d_dG, R * kpad));
  CK(cudaMemset(h->d_dG, 0, R * kpad * sizeof(float)));
  if (h->aev_aliased) {
    h->d_aev = h->d_dG;
  } else {
    CK(cudaMalloc(&h->d_aev, R * kpad * sp * es));
    CK(cudaMemset(h->d_aev, 0, R * kpad * sp * es));
  }
  CK(cudaMalloc(&h->d_h1, R * h->ldh1 * es));
  CK(cudaMemset(h->d_h1, 0, R * h->ldh1 * es));
  if (h->prec == Prec::F32) {  // the tensor-core path keeps h2, z3, d3 and d2 on chip
    CK(cudaMalloc(&h->d_h2, R * h->ldh2 * es));
    CK(cudaMemset(h->d_h2, 0, R * h->ldh2 * es));
    CK(dalloc(&h->d_z3, R * h->ldz3));
    CK(cudaMemset(h->d_z3, 0, R * h->ldz3 * sizeof(float)));
    CK(cudaMalloc(&h->d_d3, R * h->ldz3 * es));
    CK(cudaMemset(h->d_d3, 0, R * h->ldz3 * es));
  }
  CK(dalloc(&h->d_y, R * M));
  CK(dalloc(&h->d_atom_e, R));
  CK(dalloc(&h->d_pos_in, (size_t)N * 3));
  CK(dalloc(&h->d_E, n_mols));
  CK(dalloc(&h->d_F, (size_t)N * 3));

  // ---- weights: pack into the product layouts ----
  // W1  [e]: rows m*h1+o, kpad cols         W2  [e][m]: rows o, 256 cols
  // W3  [e][m]: rows o, 192 cols            W3T [e][m]: rows (h2 index), 160 cols
  // W2T [e][m]: rows (h1 index), 192 cols   W1T [e]: rows kpad (feature), M*256 cols
  // Device widths hp (multiples of 32) may exceed the caller's widths: the
  // extra rows and columns stay zero.
  const float* W = params->weights;
  const long per_model = model_params(md);
  const int NE = md.ns;
  const auto& hp = md.hpad;
  long eoff[kSpecies];
  {
    long a = 0;
    for (int e = 0; e < NE; ++e) {
      eoff[e] = a;
      a += element_params(md, e);
    }
  }
  size_t rows_w1 = 0, rows_w2 = 0, rows_w3 = 0, rows_w3t = 0, rows_w2t = 0;
  for (int e = 0; e < NE; ++e) {
    rows_w1 += (size_t)M * hp[e][0];
    rows_w2 += (size_t)M * hp[e][1];
    rows_w3 += (size_t)M * hp[e][2];
    rows_w3t += (size_t)M * hp[e][1];
    rows_w2t += (size_t)M * hp[e][0];
  }
  // the forward weights of the split path hold hi | lo side by side
  const size_t ld_w1 = (size_t)sp * kpad, ld_w2 = (size_t)sp * kH1Max,
               ld_w3 = (size_t)sp * kH2Max, ld_w3t = kH3Max, ld_w2t = kH2Max,
               ld_w1t = (size_t)M * kH1Max;
  h->w_off[0] = 0;
  h->w_off[1] = h->w_off[0] + rows_w1 * ld_w1;
  h->w_off[2] = h->w_off[1] + rows_w2 * ld_w2;
  h->w_off[3] = h->w_off[2] + rows_w3 * ld_w3;
  h->w_off[4] = h->w_off[3] + rows_w3t * ld_w3t;
  h->w_off[5] = h->w_off[4] + rows_w2t * ld_w2t;
  const size_t w_total = h->w_off[5] + (size_t)NE * kpad * ld_w1t;
  Packer pk{h->prec};
  pk.resize(w_total);
  size_t b1_total = rows_w1, b2_total = rows_w2, b3_total = rows_w3;
  std::vector<float> bias(b1_total + b2_total + b3_total, 0.f);
  std::vector<float> w4((size_t)kSpecies * kMaxModels * kH3Max, 0.f), b4((size_t)kSpecies * kMaxModels, 0.f);
  // per element/model row starts
  size_t r1[kSpecies], r2[kSpecies][kMaxModels], r3[kSpecies][kMaxModels], r3t[kSpecies][kMaxModels],
      r2t[kSpecies][kMaxModels];
  {
    size_t a1 = 0, a2 = 0, a3 = 0, a3t = 0, a2t = 0;
    for (int e = 0; e < NE; ++e) {
      r1[e] = a1;
      a1 += (size_t)M * hp[e][0];
      for (int m = 0; m < M; ++m) {
        r2[e][m] = a2;
        a2 += hp[e][1];
        r3[e][m] = a3;
        a3 += hp[e][2];
        r3t[e][m] = a3t;
        a3t += hp[e][1];
        r2t[e][m] = a2t;
        a2t += hp[e][0];
      }
    }
  }
  const int nfeat = md.nfeat;
  for (int e = 0; e < NE; ++e) {
    // caller's widths n1..n3 (weight layout), device widths p1 (row stride of W1 per member)
    const int n1 = md.hidden[e][0], n2 = md.hidden[e][1], n3 = md.hidden[e][2], p1 = hp[e][0];
    for (int m = 0; m < M; ++m) {
      const float* p = W + (size_t)m * per_model + eoff[e];
      const float *W1 = p, *b1 = W1 + (size_t)n1 * nfeat, *W2 = b1 + n1, *b2 = W2 + (size_t)n2 * n1,
                  *W3 = b2 + n2, *b3 = W3 + (size_t)n3 * n2, *w4p = b3 + n3, *b4p = w4p + n3;
      for (int o = 0; o < n1; ++o) {
        for (int k = 0; k < nfeat; ++k) {
          const float v = W1[(size_t)o * nfeat + k];
          pk.set_fwd(h->w_off[0] + (r1[e] + (size_t)m * p1 + o) * ld_w1 + k, kpad, v, h->split);
          pk.set(h->w_off[5] + ((size_t)e * kpad + k) * ld_w1t + (size_t)m * p1 + o, v);
        }
        bias[r1[e] + (size_t)m * p1 + o] = b1[o];
      }
      for (int o = 0; o < n2; ++o) {
        for (int k = 0; k < n1; ++k) {
          const float v = W2[(size_t)o * n1 + k];
          pk.set_fwd(h->w_off[1] + (r2[e][m] + o) * ld_w2 + k, kH1Max, v, h->split);
          pk.set(h->w_off[4] + (r2t[e][m] + k) * ld_w2t + o, v);
        }
        bias[b1_total + r2[e][m] + o] = b2[o];
      }
      for (int o = 0; o < n3; ++o) {
        for (int k = 0; k < n2; ++k) {
          const float v = W3[(size_t)o * n2 + k];
          pk.set_fwd(h->w_off[2] + (r3[e][m] + o) * ld_w3 + k, kH2Max, v, h->split);
          pk.set(h->w_off[3] + (r3t[e][m] + k) * ld_w3t + o, v);
        }
        bias[b1_total + b2_total + r3[e][m] + o] = b3[o];
        w4[((size_t)e * kMaxModels + m) * kH3Max + o] = w4p[o];
      }
      b4[(size_t)e * kMaxModels + m] = b4p[0];
    }
  }
  CK(cudaMalloc(&h->d_w, w_total * es));
  CK(cudaMemcpy(h->d_w, pk.data(), w_total * es, cudaMemcpyHostToDevice));
  CK(dalloc(&h->d_b, bias.size()));
  CK(cudaMemcpy(h->d_b, bias.data(), bias.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(dalloc(&h->d_w4, w4.size()));
  CK(cudaMemcpy(h->d_w4, w4.data(), w4.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(dalloc(&h->d_b4, b4.size()));
  CK(cudaMemcpy(h->d_b4, b4.data(), b4.size() * sizeof(float), cudaMemcpyHostToDevice));

  // ---- problem lists of the six matrix-product layers ----
  char* wb = static_cast<char*>(h->d_w);
  char* aev = static_cast<char*>(h->d_aev);
  char* H1 = static_cast<char*>(h->d_h1);
  char* H2 = static_cast<char*>(h->d_h2);
  float* Z3 = h->d_z3;
  char* D3 = static_cast<char*>(h->d_d3);
  const bool tc = h->prec != Prec::F32;
  const int bm = tc ? 128 : simt_tile_m(), bn_simt = simt_tile_n();
  for (int e = 0; e < NE; ++e) {
    const int Me = h->elem_count[e];
    if (Me == 0) continue;
    const int n1 = hp[e][0], n2 = hp[e][1], n3 = hp[e][2];
    const size_t row0 = h->elem_row0[e];
    {  // layer 1 forward
      GemmProblem P{};
      P.A = aev + row0 * kpad * sp * es; P.lda = (long)(kpad * sp);
      P.B = wb + (h->w_off[0] + r1[e] * ld_w1) * es; P.ldb = ld_w1;
      P.D = H1 + row0 * h->ldh1 * es; P.ldd = h->ldh1;
      P.bias = h->d_b + r1[e];
      P.M = Me; P.N = M * n1; P.K = tc ? (int)kpad : nfeat; P.epi = (int)Epi::BiasCelu;
      P.a_row0 = (int)row0; P.b_row0 = (int)r1[e]; P.elem = e; P.model = -1;
      if (h->split) {  // features, W1 and h1 as hi | lo
        P.split = 1;
        P.a_lo = (int)kpad;
        P.b_lo = (int)kpad;
        P.d_lo = M * kH1Max;
      }
      h->L[0].probs.push_back(P);
      add_tiles(h->L[0], bm, tc ? 256 : bn_simt);  // first layer forward
    }
    {  // layer 1 reverse: dE/dG = sum_m delta1_m W1_m
      GemmProblem P{};
      P.A = H1 + row0 * h->ldh1 * es; P.lda = h->ldh1;
      P.B = wb + (h->w_off[5] + (size_t)e * kpad * ld_w1t) * es; P.ldb = ld_w1t;
      P.D = h->d_dG + row0 * kpad; P.ldd = (long)kpad;
      P.M = Me; P.N = tc ? (int)kpad : nfeat; P.K = M * n1; P.epi = (int)Epi::Store;
      P.a_row0 = (int)row0; P.b_row0 = e * (int)kpad; P.elem = e; P.model = -1;
      h->L[5].probs.push_back(P);
      add_tiles(h->L[5], bm, tc ? 256 : bn_simt);
    }
    // layers 2 and 3 and their reverse as grouped products: the FP32 path only
    // (on tensor cores the fused tail keeps h2, d3 and d2 on chip)
    for (int m = 0; m < (tc ? 0 : M); ++m) {
      {  // layer 2 forward
        GemmProblem P{};
        P.A = H1 + (row0 * h->ldh1 + (size_t)m * n1) * es; P.lda = h->ldh1;
        P.B = wb + (h->w_off[1] + r2[e][m] * ld_w2) * es; P.ldb = ld_w2;
        P.D = H2 + (row0 * h->ldh2 + (size_t)m * n2) * es; P.ldd = h->ldh2;
        P.bias = h->d_b + b1_total + r2[e][m];
        P.M = Me; P.N = n2; P.K = n1; P.epi = (int)Epi::BiasCelu;
        P.a_row0 = (int)row0; P.a_col0 = m * n1; P.b_row0 = (int)r2[e][m]; P.elem = e; P.model = m;
        h->L[1].probs.push_back(P);
        add_tiles(h->L[1], bm, tc ? 256 : bn_simt);
      }
      {  // layer 3 forward: the FP32 pre-activation for k_head
        GemmProblem P{};
        P.A = H2 + (row0 * h->ldh2 + (size_t)m * n2) * es; P.lda = h->ldh2;
        P.B = wb + (h->w_off[2] + r3[e][m] * ld_w3) * es; P.ldb = ld_w3;
        P.D = Z3 + (row0 * h->ldz3 + (size_t)m * n3); P.ldd = h->ldz3;
        P.epi = (int)Epi::Bias;
        P.bias = h->d_b + b1_total + b2_total + r3[e][m];
        P.M = Me; P.N = n3; P.K = n2;
        P.a_row0 = (int)row0; P.a_col0 = m * n2; P.b_row0 = (int)r3[e][m]; P.elem = e; P.model = m;
        h->L[2].probs.push_back(P);
        add_tiles(h->L[2], bm, tc ? 256 : bn_simt);
      }
      {  // layer 3 reverse: delta2 = (delta3 W3) * celu'(h2), in place over h2
        GemmProblem P{};
        P.A = D3 + (row0 * h->ldz3 + (size_t)m * n3) * es; P.lda = h->ldz3;
        P.B = wb + (h->w_off[3] + r3t[e][m] * ld_w3t) * es; P.ldb = ld_w3t;
        P.D = H2 + (row0 * h->ldh2 + (size_t)m * n2) * es; P.ldd = h->ldh2;
        P.M = Me; P.N = n2; P.K = n3; P.epi = (int)Epi::DCelu;
        P.a_row0 = (int)row0; P.a_col0 = m * n3; P.b_row0 = (int)r3t[e][m]; P.elem = e; P.model = m;
        h->L[3].probs.push_back(P);
        add_tiles(h->L[3], bm, tc ? 256 : bn_simt);
      }
      {  // layer 2 reverse: delta1 = (delta2 W2) * celu'(h1), in place over h1
        GemmProblem P{};
        P.A = H2 + (row0 * h->ldh2 + (size_t)m * n2) * es; P.lda = h->ldh2;
        P.B = wb + (h->w_off[4] + r2t[e][m] * ld_w2t) * es; P.ldb = ld_w2t;
        P.D = H1 + (row0 * h->ldh1 + (size_t)m * n1) * es; P.ldd = h->ldh1;
        P.M = Me; P.N = n1; P.K = n2; P.epi = (int)Epi::DCelu;
        P.a_row0 = (int)row0; P.a_col0 = m * n2; P.b_row0 = (int)r2t[e][m]; P.elem = e; P.model = m;
        h->L[4].probs.push_back(P);
        add_tiles(h->L[4], bm, tc ? 256 : bn_simt);
      }
    }
  }
  if (!tc)  // the SIMT products read 16-byte vectors along K
    for (const Layer& L : h->L)
      for (const GemmProblem& P : L.probs)
        if (((reinterpret_cast<uintptr_t>(P.A) | reinterpret_cast<uintptr_t>(P.B)) & 15) || (P.lda | P.ldb) % 4 ||
            P.K % 4)
          return fail(h, NNP_ERR_UNSUPPORTED, "FP32 product operands not 16-byte aligned");
  if (tc) {
    if (tc_maps_bytes() > sizeof(h->tc_maps[0])) return fail(h, NNP_ERR_UNSUPPORTED, "tensor map size");
    CK(tc_set_smem());
    // CTA pairs for the first layer's two products (grouped products of
    // layers 2 and 3 with K <= 3 x 256 and N <= 192 ran slower on pairs:
    // fewer, longer tiles for the same work)
    h->l1_max_pairs = h->single_cta ? 0 : std::min(tc2_max_pairs(h->sms), h->sms / 2);
    h->l1_pairs = h->l1_max_pairs > 0;
    const uint64_t R64 = (uint64_t)h->n_rows;
    struct MapSpec {
      const void* base;
      uint64_t rows, cols;
    };
    const MapSpec A[6] = {{h->d_aev, R64, (uint64_t)kpad * sp},
                          {h->d_h1, R64, (uint64_t)h->ldh1},
                          {h->d_h1, R64, (uint64_t)h->ldh1},
                          {h->d_d3, R64, (uint64_t)h->ldz3},
                          {h->d_h2, R64, (uint64_t)h->ldh2},
                          {h->d_h1, R64, (uint64_t)h->ldh1}};
    const MapSpec B[6] = {{wb + h->w_off[0] * es, rows_w1, ld_w1},
                          {wb + h->w_off[1] * es, rows_w2, ld_w2},
                          {wb + h->w_off[2] * es, rows_w3, ld_w3},
                          {wb + h->w_off[3] * es, rows_w3t, ld_w3t},
                          {wb + h->w_off[4] * es, rows_w2t, ld_w2t},
                          {wb + h->w_off[5] * es, (uint64_t)NE * kpad, ld_w1t}};
    h->l1_b_base[0] = B[0].base;
    h->l1_b_rows[0] = B[0].rows;
    h->l1_b_cols[0] = B[0].cols;
    h->l1_b_base[1] = B[5].base;
    h->l1_b_rows[1] = B[5].rows;
    h->l1_b_cols[1] = B[5].cols;
    // the two first-layer products (layers 2 and 3 run in the fused tail)
    for (int l : {0, 5}) {
      if (!tc_make_map(h->tc_maps[l], A[l].base, h->prec, A[l].rows, A[l].cols, A[l].cols, 128) ||
          !tc_make_map(h->tc_maps[l] + 128, B[l].base, h->prec, B[l].rows, B[l].cols, B[l].cols,
                       (uint32_t)h->tc_box[l]))
        return fail(h, NNP_ERR_CUDA, "cuTensorMapEncodeTiled failed for layer " + std::to_string(l));
    }
    // outputs of the two first-layer products, stored by TMA: h1 (16-bit, 64-column
    // boxes) and dE/dG (FP32, 32-column boxes)
    if (!tc_make_map(h->tc_maps[0] + 256, h->d_h1, h->prec, R64, (uint64_t)h->ldh1, (uint64_t)h->ldh1, 128) ||
        !tc_make_map(h->tc_maps[5] + 256, h->d_dG, Prec::F32, R64, (uint64_t)kpad,
                     (uint64_t)kpad, 128, 32))
      return fail(h, NNP_ERR_CUDA, "cuTensorMapEncodeTiled failed for a first-layer output");
    // fused tail: one problem per (element, member), tiles of 128 rows
    for (int e = 0; e < NE; ++e) {
      const int Me = h->elem_count[e];
      if (Me == 0) continue;
      for (int m = 0; m < M; ++m) {
        TailProblem T{};
        T.Me = Me;
        T.row0 = h->elem_row0[e];
        T.h1 = hp[e][0];
        T.h2 = hp[e][1];
        T.h3 = hp[e][2];
        T.a_col0 = m * T.h1;
        T.w2_row0 = (int)r2[e][m];
        T.w3_row0 = (int)r3[e][m];
        T.w3t_row0 = (int)r3t[e][m];
        T.w2t_row0 = (int)r2t[e][m];
        T.b2 = h->d_b + b1_total + r2[e][m];
        T.b3 = h->d_b + b1_total + b2_total + r3[e][m];
        T.w4 = h->d_w4 + ((size_t)e * kMaxModels + m) * kH3Max;
        T.b4 = b4[(size_t)e * kMaxModels + m];
        T.inv_m = 1.0f / (float)M;
        T.y = h->d_y + (size_t)T.row0 * M + m;
        T.h1_lo = M * kH1Max;
        T.ldy = M;
        const int pi = (int)h->tail_probs.size();
        h->tail_probs.push_back(T);
        for (int m0 = 0; m0 < Me; m0 += 128) h->tail_tiles.push_back(GemmTile{pi, m0, 0, 0});
      }
    }
    if (tail_maps_bytes() > sizeof(h->tail_maps)) return fail(h, NNP_ERR_UNSUPPORTED, "tail map size");
    const MapSpec TW[4] = {B[1], B[2], B[3], B[4]};  // w2, w3, w3t, w2t
    if (!tc_make_map(h->tail_maps, h->d_h1, h->prec, R64, (uint64_t)h->ldh1, (uint64_t)h->ldh1, 128))
      return fail(h, NNP_ERR_CUDA, "cuTensorMapEncodeTiled failed for the fused tail");
    for (int i = 0; i < 4; ++i)
      if (!tc_make_map(h->tail_maps + 128 * (i + 1), TW[i].base, h->prec, TW[i].rows, TW[i].cols,
                       TW[i].cols, (uint32_t)tail_weight_box(i)))
        return fail(h, NNP_ERR_CUDA, "cuTensorMapEncodeTiled failed for the fused tail");
    if (!tc_make_map(h->tail_maps + 5 * 128, h->d_h1, h->prec, R64, (uint64_t)h->ldh1, (uint64_t)h->ldh1,
                     128, 32, true))
      return fail(h, NNP_ERR_CUDA, "cuTensorMapEncodeTiled failed for the fused tail");
    CK(tail_set_smem());
    {  // balance the tail's tiles by network size (two products per layer and direction)
      std::vector<double> cost;
      for (const GemmTile& t : h->tail_tiles) {
        const TailProblem& T = h->tail_probs[t.problem];
        cost.push_back((double)T.h1 * T.h2 + (double)T.h2 * T.h3);
      }
      balance_tiles(h->tail_tiles, cost, h->sms, h->tail_off);
      CK(dalloc(&h->d_tail_off, h->tail_off.size()));
      CK(cudaMemcpy(h->d_tail_off, h->tail_off.data(), sizeof(int) * h->tail_off.size(),
                    cudaMemcpyHostToDevice));
    }
    CK(dalloc(&h->d_tail_probs, h->tail_probs.size()));
    CK(dalloc(&h->d_tail_tiles, h->tail_tiles.size()));
    if (!h->tail_probs.empty()) {
      CK(cudaMemcpy(h->d_tail_probs, h->tail_probs.data(), sizeof(TailProblem) * h->tail_probs.size(),
                    cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_tail_tiles, h->tail_tiles.data(), sizeof(GemmTile) * h->tail_tiles.size(),
                    cudaMemcpyHostToDevice));
    }
  }
  for (auto& L : h->L) {
    CK(dalloc(&L.d_probs, L.probs.size()));
    CK(dalloc(&L.d_tiles, L.tiles.size()));
    if (!L.probs.empty())
      CK(cudaMemcpy(L.d_probs, L.probs.data(), sizeof(GemmProblem) * L.probs.size(), cudaMemcpyHostToDevice));
    if (!L.tiles.empty())
      CK(cudaMemcpy(L.d_tiles, L.tiles.data(), sizeof(GemmTile) * L.tiles.size(), cudaMemcpyHostToDevice));
  }

  if (h->prec != Prec::F32) {  // first-layer tiles balanced over the SMs (or SM pairs)
    const nnp_status st = set_l1_tiles(h, h->l1_bn);
    if (st != NNP_OK) return st;
  }
  h->mol_off_h.assign(mol_offsets, mol_offsets + n_mols + 1);
  h->adj_chunk = N >= 152 * 64 ? 8 * h->adj_warps : h->adj_warps;
  {
    const nnp_status st = build_work_list(h, h->adj_warps, h->adj_chunk);
    if (st != NNP_OK) return st;
  }
  CK(aev_set_smem_limits(aev_fwd_smem_bytes(cap_r, cap_a, h->fwd_warps), 0));
  CK(cudaDeviceSynchronize());
  guard.ok = true;
  *out = h;
  return NNP_OK;
}

}  // extern "C"

namespace {

void run_gemm(nnp_ctx* h, int layer, cudaStream_t s) {
  Layer& L = h->L[layer];
  if (L.tiles.empty()) return;
  if (h->prec == Prec::F32)
    launch_gemm_simt(L.d_probs, L.d_tiles, (int)L.tiles.size(), s);
  else if (h->l1_pairs && (layer == 0 || layer == 5))
    launch_gemm_tc2(L.d_probs, L.d_tiles, L.d_cta_off, (int)L.cta_off.size() - 1, h->prec,
                    h->tc_box[layer], h->tc_maps[layer], h->d_status, h->d_abort, s);
  else
    launch_gemm_tc(L.d_probs, L.d_tiles, L.d_cta_off, (int)L.cta_off.size() - 1, h->prec,
                   h->tc_box[layer], h->tc_maps[layer], h->d_status, h->d_abort, s);
}

// NVTX ranges named after the stages (nnp_stage order), around the host-side
// enqueue of each stage: a profiler that projects them onto the GPU work
// (or a timeline of the direct-launch path) shows which kernels belong to
// which stage.  They cost nothing without a tool attached.
const char* const kStageRange[NNP_NUM_STAGES] = {
    "nnp/neighbors", "nnp/features", "nnp/l1_fwd", "nnp/l2_fwd", "nnp/l3_fwd",
    "nnp/energy",    "nnp/l3_rev",   "nnp/l2_rev", "nnp/l1_rev", "nnp/adjoint"};

struct StageRanges {
  bool open = false;
  void next(int i) {  // close the current stage's range, open stage i's
    if (open) nvtxRangePop();
    open = i < NNP_NUM_STAGES;
    if (open) nvtxRangePushA(kStageRange[i]);
  }
  ~StageRanges() {
    if (open) nvtxRangePop();
  }
};

// The whole step, enqueued on s.  With ev != nullptr an event is recorded
// after each stage (ev[0] before the first); stage order is nnp_stage.
int enqueue_step(nnp_ctx* h, const float* pos, double* E, double* F, cudaStream_t s,
                 cudaEvent_t* ev = nullptr) {
  const Geometry g = h->geometry();
  int kernels = 0;
  StageRanges ranges;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], s);
    ranges.next(i);
  };
  auto gemm = [&](int layer) {
    if (!h->L[layer].tiles.empty()) ++kernels;
    run_gemm(h, layer, s);
  };
  mark(0);
  // with forces, the gather also zeroes them and the reverse pass's overflow count
  launch_gather_positions(pos, h->d_orig, h->d_species_int, h->d_pos, h->n_atoms, h->d_status, F,
                          F ? h->d_ovf : nullptr, s);
  if (h->use_cells) {
    launch_neighbors_cells(g, h->nl, h->aevc, h->cells, h->cellbuf, h->n_atoms, h->d_status, s);
    kernels += 5;  // gather, bin count, scan, fill, neighbours
  } else {
    launch_neighbors_mol(g, h->nl, h->aevc, h->d_nbr_work, h->n_nbr_work, h->max_mol, h->d_status, s);
    kernels += 2;
  }
  mark(1);
  launch_aev(g, h->nl, h->aevc, h->d_row_of_int, h->d_aev, h->prec, h->fwd_warps, s, h->split != 0);
  ++kernels;
  mark(2);
  gemm(0);
  mark(3);
  bool fork = false;
  if (h->prec != Prec::F32) {
    auto tail = [&](int reverse) {
      if (h->tail_tiles.empty()) return;
      launch_mlp_tail(h->d_tail_probs, h->d_tail_tiles, h->d_tail_off, (int)h->tail_off.size() - 1, h->prec,
                      h->tail_maps, reverse, h->d_status, h->d_abort, s);
      ++kernels;
    };
    // tensor cores: L2 fwd, L3 fwd + output layer, L3 rev, L2 rev in one
    // kernel (without forces, the forward phases); with split operands each
    // forward product as three
    tail(h->split ? (F ? 2 : 3) : (F ? 1 : 0));
    mark(4);
    mark(5);
    // with forces (and no per-stage events) the energy reduction runs on a
    // side stream, concurrently with the reverse pass, joined at the end
    cudaStream_t se = s;
    if (F && !ev) {
      fork = true;
      cudaEventRecord(h->ev_fork, s);
      cudaStreamWaitEvent(h->side, h->ev_fork, 0);
      se = h->side;
    }
    launch_energy(h->d_y, h->n_models, h->d_row_of_int, h->d_mol_off, h->n_mols, E, h->d_atom_e, se);
    if (fork) cudaEventRecord(h->ev_join, h->side);
    ++kernels;
    mark(6);
    if (!F) return kernels;
    mark(7);
    mark(8);
  } else {
    gemm(1);
    mark(4);
    gemm(2);
    int h3[kSpecies] = {0};
    for (int e = 0; e < h->md.ns; ++e) h3[e] = h->md.hpad[e][2];
    launch_head(h->d_z3, h->ldz3, h->prec, h->d_row_elem, h->d_w4, h->d_b4, h->d_d3, h->d_y,
                h->n_rows, h->n_models, h3, s);
    ++kernels;
    mark(5);
    launch_energy(h->d_y, h->n_models, h->d_row_of_int, h->d_mol_off, h->n_mols, E, h->d_atom_e, s);
    ++kernels;
    mark(6);
    if (!F) return kernels;
    gemm(3);
    mark(7);
    gemm(4);
    mark(8);
  }
  gemm(5);
  mark(9);
  launch_aev_adjoint(g, h->nl, h->aevc, h->d_row_of_int, h->d_dG, h->d_work, h->n_work, h->d_orig,
                     F, h->adj_warps, h->smem_atoms_max, h->d_ovf, h->adj_ovf_ctas, s);
  kernels += aev_adj_launches(h->nl.cap_a);
  if (fork) cudaStreamWaitEvent(s, h->ev_join, 0);
  mark(10);
  return kernels;
}

}  // namespace

namespace {
nnp_status compute_step(nnp_ctx* h, const float* pos, double* E, double* F, cudaStream_t s);
}  // namespace

extern "C" {

nnp_status nnp_compute(nnp_handle h, const float* pos, double* E, double* F, void* stream) {
  if (!h) return NNP_ERR_ARG;
  if ((!pos && h->n_atoms) || (!E && h->n_mols)) return fail(h, NNP_ERR_ARG, "null buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  h->features_overwritten = h->aev_aliased && F != nullptr;
  cudaGetLastError();  // a stale error of the caller's must not be taken for one of these launches
  if (h->abort_steps > 0) {  // tests: this step's tensor-core kernels stop at their start
    --h->abort_steps;
    CK(cudaMemsetAsync(h->d_abort, 1, sizeof(int), s));
    const nnp_status st = compute_step(h, pos, E, F, s);
    CK(cudaMemsetAsync(h->d_abort, 0, sizeof(int), s));
    return st;
  }
  return compute_step(h, pos, E, F, s);
}

}  // extern "C"

namespace {

// One evaluation: a graph replay (captured again when the buffers change) or
// direct launches.
nnp_status compute_step(nnp_ctx* h, const float* pos, double* E, double* F, cudaStream_t s) {
  if (h->use_graph) {
    if (!h->gexec || h->g_pos != pos || h->g_E != E || h->g_F != F) {
      if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      enqueue_step(h, pos, E, F, h->cap_stream);
      const cudaError_t le = cudaGetLastError();
      const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
      if (le != cudaSuccess || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(h, NNP_ERR_CUDA, std::string("graph capture: ") +
                                         cudaGetErrorString(le != cudaSuccess ? le : ce));
      }
      const cudaError_t ie = cudaGraphInstantiate(&h->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        h->gexec = nullptr;
        return fail(h, NNP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
      }
      h->g_pos = pos;
      h->g_E = E;
      h->g_F = F;
    }
    CK(cudaGraphLaunch(h->gexec, s));
    return NNP_OK;
  }
  enqueue_step(h, pos, E, F, s);
  CK(cudaGetLastError());
  return NNP_OK;
}

}  // namespace

namespace nnp {
int enqueue_nnp(nnp_ctx* h, const float* pos, double* E, double* F, cudaStream_t s) {
  const int k = enqueue_step(h, pos, E, F, s);
  return cudaGetLastError() == cudaSuccess ? k : -1;
}
void handle_shape(const nnp_ctx* h, int* n_atoms, int* n_mols, std::vector<int>& mol_off) {
  *n_atoms = h->n_atoms;
  *n_mols = h->n_mols;
  mol_off = h->mol_off_h;
}
void set_last_stream(nnp_ctx* h, cudaStream_t s) { h->last_stream = s; }
}  // namespace nnp

extern "C" {

nnp_status nnp_compute_timed(nnp_handle h, const float* pos, double* E, double* F, void* stream,
                              float* stage_ms, int32_t n_stages) {
  if (!h || !stage_ms || n_stages < NNP_NUM_STAGES) return NNP_ERR_ARG;
  if ((!pos && h->n_atoms) || (!E && h->n_mols)) return fail(h, NNP_ERR_ARG, "null buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  cudaEvent_t ev[NNP_NUM_STAGES + 1];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  enqueue_step(h, pos, E, F, s, ev);
  const int last = F ? NNP_NUM_STAGES : NNP_STAGE_ENERGY + 1;
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaEventSynchronize(ev[last]);
  for (int i = 0; i < NNP_NUM_STAGES; ++i) {
    stage_ms[i] = 0.f;
    if (err == cudaSuccess && i < last) cudaEventElapsedTime(&stage_ms[i], ev[i], ev[i + 1]);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  CK(err);
  return NNP_OK;
}

int32_t nnp_kernels_per_step(nnp_handle h, int32_t with_forces) {
  if (!h) return -1;
  int k = (h->use_cells ? 5 : 2) + 1 + 1;  // gather (+ cell binning), neighbours, features, energy
  k += h->L[0].tiles.empty() ? 0 : 1;
  if (h->prec == Prec::F32) {
    k += 1;  // head
    for (int l = 1; l < 3; ++l) k += h->L[l].tiles.empty() ? 0 : 1;
    if (with_forces)
      for (int l = 3; l < 5; ++l) k += h->L[l].tiles.empty() ? 0 : 1;
  } else {
    k += h->tail_tiles.empty() ? 0 : 1;
  }
  if (with_forces)  // L1 reverse, featurizer reverse (main and overflow launches)
    k += aev_adj_launches(h->nl.cap_a) + (h->L[5].tiles.empty() ? 0 : 1);
  return k;
}

nnp_status nnp_autotune(nnp_handle h, const float* pos, void* stream, int32_t* chosen) {
  if (!h || (!pos && h->n_atoms)) return NNP_ERR_ARG;
  if (h->n_atoms == 0) return NNP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* dE = nullptr;
  double* dF = nullptr;
  CK(dalloc(&dE, h->n_mols));
  CK(dalloc(&dF, 3 * (size_t)h->n_atoms));
  float ms[NNP_NUM_STAGES];
  auto time_stages = [&](int a, int b) -> float {  // median of 9 of stages [a, b]
    float t[9];
    for (int r = 0; r < 9; ++r) {
      if (nnp_compute_timed(h, pos, dE, dF, stream, ms, NNP_NUM_STAGES) != NNP_OK) return 1e30f;
      t[r] = 0.f;
      for (int k = a; k <= b; ++k) t[r] += ms[k];
    }
    std::sort(t, t + 9);
    return t[4];
  };
  // warm-up: the first candidates must not be timed while clocks and caches settle
  for (int r = 0; r < 10; ++r)
    if (nnp_compute_timed(h, pos, dE, dF, stream, ms, NNP_NUM_STAGES) != NNP_OK) break;
  nnp_status st = NNP_OK;
  // featurizer: atoms (warps) per CTA
  {
    int best = h->fwd_warps;
    float best_t = 1e30f;
    for (int w : {2, 4, 8}) {
      if (aev_set_smem_limits(aev_fwd_smem_bytes(h->nl.cap_r, h->nl.cap_a, w), 0) != cudaSuccess) continue;
      h->fwd_warps = w;
      const float t = time_stages(NNP_STAGE_FEATURES, NNP_STAGE_FEATURES);
      if (t < best_t) {
        best_t = t;
        best = w;
      }
    }
    h->fwd_warps = best;
  }
  // reverse pass: warps per CTA and centres per work item
  {
    int bw = h->adj_warps, bc = h->adj_chunk, bs = h->adj_shared_acc;
    float best_t = 1e30f;
    for (int sh : {1, 0})
      for (int w : {2, 4})
        for (int mult : {1, 4, 8}) {
          if (build_work_list(h, w, mult * w, sh) != NNP_OK) continue;
          const float t = time_stages(NNP_STAGE_ADJOINT, NNP_STAGE_ADJOINT);
          if (t < best_t) {
            best_t = t;
            bw = w;
            bc = mult * w;
            bs = sh;
          }
        }
    st = build_work_list(h, bw, bc, bs);
  }
  // first layer: N tile of the tensor-core products
  if (st == NNP_OK && h->prec != Prec::F32) {
    int best = h->l1_bn;
    float best_t = 1e30f;
    for (int bn : {256, 128}) {
      if (set_l1_tiles(h, bn) != NNP_OK) continue;
      const float t = time_stages(NNP_STAGE_L1_FWD, NNP_STAGE_L1_FWD) +
                      time_stages(NNP_STAGE_L1_REV, NNP_STAGE_L1_REV);
      if (t < best_t) {
        best_t = t;
        best = bn;
      }
    }
    st = set_l1_tiles(h, best);
  }
  cudaStreamSynchronize(s);
  cudaFree(dE);
  cudaFree(dF);
  if (h->gexec) {  // the schedule changed: capture again on next use
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  if (chosen) {
    chosen[0] = h->fwd_warps;
    chosen[1] = h->adj_warps;
    chosen[2] = h->adj_chunk;
    chosen[3] = h->l1_bn;
    chosen[4] = h->adj_shared_acc;
  }
  return st;
}

nnp_status nnp_set_schedule(nnp_handle h, const int32_t* schedule) {
  if (!h || !schedule) return NNP_ERR_ARG;
  const int fw = schedule[0], aw = schedule[1], ac = schedule[2], bn = schedule[3], sh = schedule[4];
  const bool fw_ok = fw == 2 || fw == 4 || fw == 8;
  const bool adj_ok = (aw == 2 || aw == 4) && ac >= aw && ac <= 64 && ac % aw == 0 && (sh == 0 || sh == 1);
  const bool bn_ok = bn == 256 || bn == 128;
  if (!fw_ok || !adj_ok || !bn_ok) return fail(h, NNP_ERR_ARG, "schedule out of range");
  if (h->n_atoms == 0) return NNP_OK;
  CK(aev_set_smem_limits(aev_fwd_smem_bytes(h->nl.cap_r, h->nl.cap_a, fw), 0));
  h->fwd_warps = fw;
  nnp_status st = build_work_list(h, aw, ac, sh);
  if (st == NNP_OK && h->prec != Prec::F32) st = set_l1_tiles(h, bn);
  if (h->gexec) {  // the schedule changed: capture again on next use
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return st;
}

nnp_status nnp_compute_host(nnp_handle h, const float* pos, double* E, double* F, void* stream) {
  if (!h) return NNP_ERR_ARG;
  if ((!pos && h->n_atoms) || (!E && h->n_mols)) return fail(h, NNP_ERR_ARG, "null buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t N = h->n_atoms;
  if (N) CK(cudaMemcpyAsync(h->d_pos_in, pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, s));
  const nnp_status st = nnp_compute(h, h->d_pos_in, h->d_E, F ? h->d_F : nullptr, stream);
  if (st != NNP_OK) return st;
  if (h->n_mols) CK(cudaMemcpyAsync(E, h->d_E, sizeof(double) * h->n_mols, cudaMemcpyDeviceToHost, s));
  if (F && N) CK(cudaMemcpyAsync(F, h->d_F, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return NNP_OK;
}

nnp_status nnp_get_status(nnp_handle h) {
  if (!h) return NNP_ERR_ARG;
  CK(cudaStreamSynchronize(h->last_stream));
  unsigned st = 0;
  CK(cudaMemcpy(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CK(cudaMemset(h->d_status, 0, sizeof(unsigned)));
  if (st & kStatTimeout) return fail(h, NNP_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
  if (st & kStatNonFinite) return fail(h, NNP_ERR_NONFINITE, "non-finite position");
  if (st & (kStatCapRadial | kStatCapAngular))
    return fail(h, NNP_ERR_CAPACITY, (st & kStatCapRadial) ? "radial neighbour capacity exceeded"
                                                           : "angular neighbour capacity exceeded");
  return NNP_OK;
}

nnp_status nnp_get_capacity(nnp_handle h, int32_t* r, int32_t* a) {
  if (!h || !r || !a) return NNP_ERR_ARG;
  *r = h->nl.cap_r;
  *a = h->nl.cap_a;
  return NNP_OK;
}

nnp_status nnp_get_neighbors(nnp_handle h, int32_t kind, int32_t* counts, int32_t* lists, int32_t cap,
                             void* stream) {
  if (!h || (kind != 0 && kind != 1)) return NNP_ERR_ARG;
  if (cap < (kind == 0 ? h->nl.cap_r : h->nl.cap_a)) return fail(h, NNP_ERR_ARG, "cap too small");
  if (h->n_atoms && (!counts || !lists)) return fail(h, NNP_ERR_ARG, "null buffer");
  launch_export_neighbors(h->nl, kind, h->d_orig, h->n_atoms, counts, lists, cap,
                          static_cast<cudaStream_t>(stream));
  CK(cudaGetLastError());
  return NNP_OK;
}

nnp_status nnp_get_features(nnp_handle h, float* out, void* stream) {
  if (!h) return NNP_ERR_ARG;
  if (h->n_atoms && !out) return fail(h, NNP_ERR_ARG, "null buffer");
  if (h->features_overwritten)
    return fail(h, NNP_ERR_UNSUPPORTED,
                "recompute_aev: the last step's reverse pass reused the features' buffer");
  launch_export_features(h->d_aev, h->prec, h->d_row_of_int, h->d_orig, h->n_atoms, h->md.nfeat,
                         h->md.kpad, out, static_cast<cudaStream_t>(stream), h->split != 0);
  CK(cudaGetLastError());
  return NNP_OK;
}

nnp_status nnp_get_atomic_energies(nnp_handle h, double* out, void* stream) {
  if (!h) return NNP_ERR_ARG;
  if (h->n_atoms && !out) return fail(h, NNP_ERR_ARG, "null buffer");
  launch_export_atomic_energies(h->d_atom_e, h->d_row_of_int, h->d_orig, h->n_atoms, out,
                                static_cast<cudaStream_t>(stream));
  CK(cudaGetLastError());
  return NNP_OK;
}

}  // extern "C"
