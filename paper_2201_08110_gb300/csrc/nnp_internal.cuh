// nnp_internal.cuh -- shared declarations of the libnnp CUDA translation units.
//
// Data layout in device memory (see the C ABI in include/nnp.h):
//   * caller order: atoms as passed to nnp_create_batch, molecule-contiguous.
//   * internal order ("A"): molecule-contiguous, atoms of a molecule sorted by
//     element (stable).  Neighbour lists hold internal indices, so a list
//     ascending in internal index is grouped by element.
//   * row order ("B"): element-major (all H of the batch, then all C, ...),
//     molecule order inside an element.  The features, the network
//     activations and dE/dG are stored as rows in this order, so each
//     element's atoms form one contiguous block for the matrix products.
#pragma once

#include <utility>
#include <vector>

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

struct nnp_ctx;

namespace nnp {

// Two models share the library: ANI-2x (model 0: H, C, N, O, F, S, Cl; 8
// distance x 4 angle shifts per angular block) and ANI-1x (model 1: H, C, N,
// O; 4 x 8).  Both have 16 radial shifts and 32 features per angular block;
// each model's features are stored in its own layout (radial species-major,
// then the species-pair blocks of the row-major upper triangle).  The sizes
// below are those of ANI-2x, the larger model: they bound both.
constexpr int kSpecies = 7;
constexpr int kShfR = 16;
constexpr int kShfA = 8;
constexpr int kShfZ = 4;
constexpr int kMaxShfA = 8, kMaxShfZ = 8;               // angular shift grids of either model
constexpr int kRadial = kSpecies * kShfR;               // 112
constexpr int kPairBlocks = kSpecies * (kSpecies + 1) / 2;  // 28
constexpr int kAngPerBlock = kShfA * kShfZ;             // 32
constexpr int kAngular = kPairBlocks * kAngPerBlock;    // 896
constexpr int kFeatures = kRadial + kAngular;           // 1008
constexpr int kFeaturesPad = 1024;                      // K of the first layer, padded
constexpr int kModels = 2;

// Shape of one model's featurizer output: NS elements, NA distance shifts and
// 32 / NA angle shifts per angular block; the feature row of the first
// layer's product holds kPad >= kFeat columns (a multiple of 64, the
// tensor-core K box).  kZetaInt: the angular exponent Zeta when it is an
// integer the kernels raise to by repeated multiplication (ANI-1x: 32), else
// 0 (ANI-2x: Zeta = 14.1, taken through log2 and exp2).
template <int NS_, int NA_, int ZI_> struct AevShape {
  static constexpr int NS = NS_, NA = NA_, NZ = 32 / NA_, kZetaInt = ZI_;
  static constexpr int kRad = NS * kShfR;
  static constexpr int kNP = NS * (NS + 1) / 2;
  static constexpr int kFeat = kRad + kNP * 32;
  static constexpr int kPad = (kFeat + 63) / 64 * 64;
};
using ShapeANI2x = AevShape<7, 8, 0>;   // 1008 features, rows of 1024
using ShapeANI1x = AevShape<4, 4, 32>;  // 384 features
static_assert(ShapeANI2x::kFeat == kFeatures && ShapeANI2x::kPad == kFeaturesPad, "ANI-2x layout");
static_assert(ShapeANI1x::kFeat == 384 && ShapeANI1x::kPad == 384, "ANI-1x layout");

// Host description of a model: elements, widths of the caller's weights, the
// widths the device networks use (rounded up to multiples of 32 with zero
// weights and biases: a padded unit is celu(0) = 0 and feeds nothing, so the
// energy and forces are unchanged), feature counts.
struct ModelDesc {
  int id;
  int ns, na, nz;
  int nfeat, kpad;
  int z[kSpecies];
  int hidden[kSpecies][3];  // caller's widths
  int hpad[kSpecies][3];    // device widths
  float Rcr, Rca;
};
bool model_desc(int id, ModelDesc& md);
constexpr int kMaxModels = 16;
constexpr int kRowAlign = 128;                          // row padding of every element block

// Device status bits (sticky until nnp_get_status reads them).
constexpr unsigned kStatNonFinite = 1u << 0;
constexpr unsigned kStatCapRadial = 1u << 1;
constexpr unsigned kStatCapAngular = 1u << 2;
constexpr unsigned kStatTimeout = 1u << 3;

// Hidden widths per element (H, C, N, O, F, S, Cl).
constexpr int kHidden[kSpecies][3] = {{256, 192, 160}, {224, 192, 160}, {192, 160, 128},
                                      {192, 160, 128}, {160, 128, 96},  {160, 128, 96},
                                      {160, 128, 96}};
constexpr int kH1Max = 256, kH2Max = 192, kH3Max = 160;

// Featurizer constants in FP32, as the kernels use them.
struct AevConst {
  float Rcr, Rca, Rcr2, Rca2;  // cutoffs and squares (FP32)
  double Rcr2d, Rca2d;         // FP64 squares of the FP32 cutoffs (exact predicate)
  float EtaR, EtaA, Zeta;
  float ShfR[kShfR], ShfA[kMaxShfA], cosZ[kMaxShfZ], sinZ[kMaxShfZ];
  // exp(-Eta (r - Shf)^2) = 2^(-y^2) with y = sqEta r - ShfS = sqEta (r - Shf),
  // sqEta = sqrt(Eta log2(e)); gradX = -2 Eta / sqEta turns y into d/dr.
  // sqEta and ShfS are held as FP32 pairs hi + lo (the *l members), y =
  // fma(r, sqEta, -ShfS) + fma(r, sqEtal, -ShfSl): rounding them to single
  // FP32 values would shift y by up to 3e-6 for every pair alike, a bias of
  // up to 1e-5 on the features in a Gaussian's flank.
  float sqEtaR, sqEtaA, ShfRs[kShfR], ShfAs[kMaxShfA], gradR, gradA;
  float sqEtaRl, sqEtaAl, ShfRsl[kShfR], ShfAsl[kMaxShfA];
  // the same halved (the angular distance is (r_j + r_k) / 2), and
  // 0.95 Zeta (d cos' / d cos times the exponent)
  float hsqEtaA, hgradA, dcosA, hsqEtaAl;
  int pair_index[kSpecies][kSpecies];
  float box[3];
  double boxd[3];
  int periodic;
  int model;  // 0 ANI-2x, 1 ANI-1x: selects the featurizer's shape
};

// Geometry of one step: what the featurizer and its reverse pass read.
struct Geometry {
  const float4* pos;      // [N] internal order; w holds the element index (int bits)
  const int* mol_start;   // [N] first internal index of the atom's molecule
  const int* mol_end;     // [N] one past the last
  const int* species;     // [N] element index of internal atom
  int n_atoms;
};

// Lists hold internal indices in ascending order.  The featurizer relies on
// the internal order being element-sorted within each molecule: every list is
// then grouped by element, elements in ascending order.
struct NeighborLists {
  int* cnt_r;   // [N]
  int* nbr_r;   // [N][cap_r] internal indices, ascending
  int* cnt_a;   // [N]
  int* nbr_a;   // [N][cap_a] internal indices, ascending (subset of the radial list)
  int cap_r, cap_a;
};

// Cell list of one periodic region.
constexpr int kCellMaxAtoms = 32768;  // bitmask compaction limit (8 KB of masks per warp)
struct CellGrid {
  int n[3];  // cells per dimension, edge = box / n > Rcr
};
struct CellBuffers {
  int* cell_of;  // [N]
  int* count;    // [ncell]
  int* start;    // [ncell + 1]
  int* fill;     // [ncell]
  int* atoms;    // [N] atoms grouped by cell
};
bool cell_grid(const AevConst& c, int region_atoms, CellGrid& cg);
size_t cell_smem_bytes(int region_atoms);
cudaError_t cell_set_smem(size_t bytes);

// Element precision of the network activations and operands.
enum class Prec { F32 = 0, BF16 = 1, F16 = 2 };

// One matrix product D[M, N] = A[M, K] * B[N, K]^T (both K-major) with an
// epilogue.  Rows are atoms, A and D share the row index.
enum class Epi : int {
  BiasCelu = 0,   // D = celu(acc + bias[n])           (forward hidden layer)
  Bias = 1,       // D = acc + bias[n], FP32 output     (pre-activation of the last hidden layer)
  DCelu = 2,      // D = acc * celu'(D_in-place)       (reverse through a hidden layer)
  Store = 3       // D = acc (FP32 output)              (dE/dG)
};

struct GemmProblem {
  const void* A;  long lda;   // element offset already applied
  const void* B;  long ldb;
  void* D;        long ldd;
  const float* bias;
  int M, N, K;
  int epi;
  int a_row0, b_row0, a_col0, b_col0, d_col0;  // used by the tensor-core path (TMA coordinates)
  int elem, model;
  // Tensor-core path, split operands: with split = 1 the product is
  // A_hi B_hi + A_lo B_hi + A_hi B_lo, the lo halves a_lo / b_lo columns to the
  // right of the hi halves in the same arrays; with d_lo > 0 a 16-bit output
  // is stored as hi = round(v) and lo = round(v - hi), lo d_lo columns right.
  int split, a_lo, b_lo, d_lo;
};

// The fused tail of one (element, ensemble member): second and third hidden
// layers, output layer and their reverse pass (tensor-core path).
struct TailProblem {
  int Me;       // atoms of the element
  int row0;     // first row of the element block
  int h1, h2, h3;
  int a_col0;   // first column of this member in the h1 activations
  int w2_row0, w3_row0, w3t_row0, w2t_row0;  // rows in the stacked weight arrays
  const float* b2;
  const float* b3;
  const float* w4;
  float b4, inv_m;
  float* y;     // y + row0 * M + member, stride ldy
  long ldy;
  int h1_lo;    // split mode: columns from h1_hi to h1_lo (M * 256)
};

// A tile of the flattened problem list.
struct GemmTile {
  int problem, m0, n0;
  int width;  // columns of the tile; 0: the weight box's rows (clipped to N)
};

// Launch with programmatic stream serialization: the kernel may start while
// the previous kernel in the stream finishes; it waits (griddepcontrol.wait)
// before touching that kernel's results.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---- kernels' host launchers ------------------------------------------------

// F_zero / ovf_zero (or null): forces and the reverse pass's overflow count
// to zero in the same launch.
// pos_int[q] = (x, y, z, element index of q as int bits)
void launch_gather_positions(const float* pos_caller, const int* orig_of_int, const int* species_int,
                             float4* pos_int, int n, unsigned* status, double* F_zero, int* ovf_zero,
                             cudaStream_t s);
// Neighbour search by work items (a0, molecule atoms, first centre, end centre),
// chunks of nbr_chunk() centres of one molecule, one CTA each.
int nbr_chunk();
size_t nbr_smem_bytes(int max_mol);
cudaError_t nbr_set_smem(size_t bytes);
void launch_neighbors_mol(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                          const int4* work, int n_work, int max_mol, unsigned* status, cudaStream_t s);
void launch_neighbors(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                      unsigned* status, cudaStream_t s);
void launch_neighbors_cells(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                            const CellGrid& cg, const CellBuffers& cb, int region_atoms,
                            unsigned* status, cudaStream_t s);
// split: 16-bit features as hi | lo rows of 2 x 1024 columns
void launch_aev(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                const int* row_of_int, void* aev_out, Prec out_prec, int warps_per_cta,
                cudaStream_t s, bool split = false);
// Reverse pass: a main launch over the work items, plus, when cap_a exceeds
// the main launch's staging capacity, a second launch for the centres with
// more angular neighbours (ovf: DEVICE int[n_atoms + 1] scratch).
void launch_aev_adjoint(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                        const int* row_of_int, const float* dG, const int4* work, int n_work,
                        const int* orig, double* F, int warps, int mol_atoms_smem_max, int* ovf,
                        int ovf_ctas, cudaStream_t s);
int aev_adj_stage_cap(int cap_a);  // main launch's per-warp staging capacity
// CTAs of the overflow launch: as many as the SMs hold at once (the launch's
// shared memory must already be allowed: aev_set_smem_limits)
int aev_adj_overflow_ctas(int cap_r, int cap_a, int warps, int model);
int aev_adj_launches(int cap_a);   // kernels per reverse pass
// dynamic shared memory to allow for both launches of the reverse pass
size_t aev_adj_launch_smem(int cap_r, int cap_a, int warps, int mol_atoms_smem_max);
// h3: width of the last hidden layer of each element (device networks)
void launch_head(const float* z3, long ldz, Prec prec, const int* row_elem, const float* w4,
                 const float* b4, void* delta3, float* y, int n_rows, int n_models,
                 const int h3[kSpecies], cudaStream_t s);
void launch_energy(const float* y, int n_models, const int* row_of_int, const int* mol_off,
                   int n_mols, double* energy_out, double* atom_energy_row, cudaStream_t s);
// FP32 grouped products on the SIMT pipes; tiles of simt_tile_m() x
// simt_tile_n() outputs.
void launch_gemm_simt(const GemmProblem* d_problems, const GemmTile* d_tiles, int n_tiles,
                      cudaStream_t s);
int simt_tile_m();
int simt_tile_n();
size_t aev_fwd_smem_bytes(int cap_r, int cap_a, int warps);
size_t aev_adj_smem_bytes(int cap_r, int cap_a, int warps, int mol_atoms_smem_max);
cudaError_t aev_set_smem_limits(size_t fwd_bytes, size_t adj_bytes);

// Inspection helpers.
void launch_export_neighbors(const NeighborLists& nl, int kind, const int* orig_of_int, int n,
                             int* counts_out, int* lists_out, int cap_out, cudaStream_t s);
// rows of kpad columns (split: hi | lo, 2 x kpad columns, exported as hi +
// lo); the first nfeat columns are exported
void launch_export_features(const void* aev, Prec prec, const int* row_of_int,
                            const int* orig_of_int, int n, int nfeat, int kpad, float* out,
                            cudaStream_t s, bool split = false);
void launch_export_atomic_energies(const double* atom_energy_row, const int* row_of_int,
                                   const int* orig_of_int, int n, double* out, cudaStream_t s);

size_t tail_maps_bytes();
int tail_weight_box(int which);  // box rows of the w2, w3, w3t, w2t maps
cudaError_t tail_set_smem();
// reverse: 0 forward only, 1 forward and reverse (one product per layer);
// with split operands (h1 stored as hi | lo, three products per forward
// layer) 2 forward and reverse, 3 forward only.  abort_req: DEVICE int read at
// kernel start; nonzero makes the kernel stop before it issues any copy or
// product, as after a bounded wait that gave up
void launch_mlp_tail(const TailProblem* probs, const GemmTile* tiles, const int* cta_off, int n_ctas,
                     Prec p, const void* maps, int reverse, unsigned* status, const int* abort_req,
                     cudaStream_t s);

// Featurizer constants (cutoffs, shift grids, species-pair table, box) of a
// model (0 ANI-2x, 1 ANI-1x).
void aev_constants(AevConst& c, const double box[3], int model = 0);

// For the MD loop (md.cu): one evaluation of a handle enqueued on s as direct
// launches (captured by the caller's graph); returns the number of kernels,
// negative if a launch failed.  The handle's atom and molecule counts and its
// molecule offsets (caller order).  The stream that nnp_get_status waits on.
int enqueue_nnp(nnp_ctx* h, const float* pos, double* E, double* F, cudaStream_t s);
void handle_shape(const nnp_ctx* h, int* n_atoms, int* n_mols, std::vector<int>& mol_off);
void set_last_stream(nnp_ctx* h, cudaStream_t s);

// Setup kernels (create time).
void launch_species_setup(const int* Z_caller, const int* mol_off, int n_mols, int n_atoms,
                          int* species_caller, int* mol_species_count, unsigned* bad,
                          cudaStream_t s);
void launch_species_place(const int* species_caller, const int* mol_off, int n_mols,
                          const int* mol_species_prefix, const int* elem_mol_prefix,
                          const int* elem_row0, int* orig_of_int, int* row_of_int,
                          int* species_int, int* mol_start, int* mol_end, int* row_elem,
                          cudaStream_t s);

}  // namespace nnp
