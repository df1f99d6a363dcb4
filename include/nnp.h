/*
 * nnp.h -- C ABI of libnnp: energy and forces of an ANI-2x-style neural
 * network potential on the NNP region, computed on one GB300 (sm_103a).
 *
 * What the library computes is the NNP term of the paper's Eq. 1,
 * V_NNP(Z, r) (Eq. 2), together with the forces F = -grad V_NNP (Eq. 3), for
 * neutral molecules (Sec. 1: "only neutral molecules"), with the ANI
 * featurizer (Sec. 1: modified Behler-Parrinello symmetry functions, 5.1 A
 * cutoff, elements H C N O F S Cl) and an ensemble of M atomic networks
 * (Sec. 2 "Optimization": 8 networks, evaluated in parallel over networks
 * and atoms).  An MD engine adds the returned energy and forces to its MM
 * terms.  Positions, energies and forces stay on the GPU (Sec. 2
 * "Optimization", first point); nnp_compute takes device pointers and a
 * stream and never synchronises or allocates.
 *
 * Featurizer (per atom i, neighbours j, k of the same molecule / periodic
 * region; the paper names it but prints no formula, this is the ANI form):
 *   fc(r; Rc) = 0.5 cos(pi r / Rc) + 0.5 for r < Rc
 *   radial  G_i[s, k] = sum_{s(j)=s, r_ij<Rcr} 1/4 exp(-EtaR (r_ij-ShfR_k)^2) fc(r_ij; Rcr)
 *   angular G_i[p(s,t), a, z] = sum_{j<k in the Rca shell} 2 ((1 + cos(theta'-ShfZ_z))/2)^Zeta
 *            exp(-EtaA ((r_ij+r_ik)/2 - ShfA_a)^2) fc(r_ij; Rca) fc(r_ik; Rca),
 *            theta' = acos(0.95 cos angle_jik)
 *   Rcr = 5.1 A, EtaR = 19.7, ShfR = 16 points 0.8..4.9 A; Rca = 3.5 A,
 *   EtaA = 12.5, Zeta = 14.1, ShfA = 8 points 0.8..3.1 A, ShfZ = 4 points
 *   0.39..2.75 rad; 1008 features = 7x16 radial + 28x8x4 angular.
 * Networks (per element; CELU alpha 0.1):
 *   H 1008-256-192-160-1, C 1008-224-192-160-1, N and O 1008-192-160-128-1,
 *   F, S and Cl 1008-160-128-96-1.  E_mol = (1/M) sum_m sum_i y_m(i).
 *
 * Units: positions in Angstrom; energy in the units of the network output;
 * forces are -dE/dx in energy units per Angstrom.
 *
 * Threading: a handle may be used by one host thread at a time.  Calls on
 * different handles are independent.
 */
#ifndef NNP_H_
#define NNP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nnp_ctx* nnp_handle;

typedef enum {
  NNP_OK = 0,
  NNP_ERR_ARG = 1,        /* bad argument (null pointer, size, layout) */
  NNP_ERR_SPECIES = 2,    /* atomic number outside the model's elements ({1, 6, 7, 8, 9, 16,
                             17} for ANI-2x, {1, 6, 7, 8} for ANI-1x) */
  NNP_ERR_CHARGE = 3,     /* total charge != 0: the model handles neutral molecules only */
  NNP_ERR_ALLOC = 4,      /* device or host allocation failed */
  NNP_ERR_CUDA = 5,       /* a CUDA call failed; see nnp_last_error */
  NNP_ERR_CAPACITY = 6,   /* device: a neighbour list exceeded its capacity */
  NNP_ERR_NONFINITE = 7,  /* device: a position was NaN or infinite */
  NNP_ERR_TIMEOUT = 8,    /* device: a bounded wait inside a kernel gave up */
  NNP_ERR_UNSUPPORTED = 9, /* the requested mode is not available */
  NNP_ERR_TOO_LARGE = 10   /* nnp_features_static: more than NNP_STATIC_MAX_ATOMS atoms */
} nnp_status;

/* Arithmetic of the networks' matrix products.  The featurizer, the neighbour
 * distances and the reverse pass to coordinates are always FP32; per-molecule
 * energies and per-atom forces are accumulated in FP64.
 *
 * With 16-bit networks each forward product is, by default, taken as three
 * tensor-core products of split operands: every FP32 value x (feature,
 * activation, weight) is held as hi = round16(x) and lo = round16(x - hi), and
 * A B = A_hi B_hi + A_lo B_hi + A_hi B_lo with FP32 accumulation (the dropped
 * A_lo B_lo is at most 2^-18 of |A||B| for BF16).  A single 16-bit rounding
 * of the weights shifts every atom of an element the same way, so its energy
 * error adds up coherently over a molecule and, where the atomic energies of a
 * molecule cancel, exceeds 2e-3 of |E|; the split forward does not.  The
 * reverse pass (forces) takes one 16-bit product per layer.  single_pass = 1
 * (nnp_params) selects one product per forward layer as well: a third of the
 * forward products, energy error up to about 6e-3 of sum_i |E_i| (BF16) or
 * 6e-4 (FP16). */
typedef enum {
  NNP_FP32 = 0, /* SIMT FP32 FMA */
  NNP_BF16 = 1, /* tensor cores (tcgen05), BF16 operands, FP32 accumulation */
  NNP_FP16 = 2  /* tensor cores (tcgen05), FP16 operands, FP32 accumulation */
} nnp_precision;

/* The two ANI models (Sec. 1; Sec. 3 "Extensibility with other NNPs" runs
 * ANI-1x beside ANI-2x).  Both: radial features of 16 shifts per element,
 * angular features of 32 per unordered element pair, layout [radial,
 * element-major | angular, pair blocks of the row-major upper triangle, each
 * distance-shift-major]; networks of three CELU (alpha 0.1) hidden layers and
 * one output per element.
 *   ANI-2x: H, C, N, O, F, S, Cl; cutoffs 5.1 / 3.5 A; 8 distance x 4 angle
 *           shifts; 1008 features; widths H 256-192-160, C 224-192-160, N and
 *           O 192-160-128, F, S and Cl 160-128-96.
 *   ANI-1x: H, C, N, O; cutoffs 5.2 / 3.5 A; 4 distance x 8 angle shifts; 384
 *           features; widths H 160-128-96, C 144-112-96, N and O 128-112-96. */
typedef enum {
  NNP_MODEL_ANI2X = 0,
  NNP_MODEL_ANI1X = 1
} nnp_model;

typedef struct {
  int32_t n_models;       /* ensemble size M >= 1 (8 for ANI-2x and ANI-1x) */
  int32_t precision;      /* nnp_precision */
  const float* weights;   /* HOST pointer, FP32, copied at create time.  Packed
                             [model][element, in the model's order][W1 b1 W2 b2 W3 b3 w4 b4],
                             each W row-major [out][in] */
  int64_t n_weights;      /* number of floats in weights; must equal
                             n_models * nnp_weights_per_model_of(model) */
  double box[3];          /* 0,0,0: non-periodic; else orthorhombic periodic box edges
                             in Angstrom (each more than twice the radial cutoff),
                             minimum-image convention */
  int32_t total_charge;   /* must be 0 */
  int32_t max_neighbors;  /* radial neighbour capacity per atom; 0 = automatic */
  int32_t max_angular;    /* angular (3.5 A) neighbour capacity per atom; 0 = automatic */
  int32_t use_graph;      /* 1: replay the step as one CUDA graph (captured on first use
                             for a given set of buffer pointers) */
  int32_t neighbor_mode;  /* 0: automatic (cell list for one periodic region of more than
                             1024 atoms, else all pairs of each molecule); 1: all pairs;
                             2: cell list (one periodic region of at most 32768 atoms,
                             else NNP_ERR_UNSUPPORTED) */
  int32_t single_pass;    /* 16-bit networks: 0 = three split-operand products per forward
                             layer (default; see nnp_precision), 1 = one product */
  int32_t recompute_aev;  /* 1: the features live only between the featurizer and the first
                             layer, in the buffer that later holds dE/dG (one fewer
                             [rows][features]-sized buffer); the reverse pass recomputes every
                             geometric quantity from the positions either way.
                             nnp_get_features then needs an energy-only nnp_compute
                             (forces_out NULL) before it, else NNP_ERR_UNSUPPORTED */
  int32_t test_abort;     /* tests only, else 0: 1 = every tensor-core kernel starts as if
                             one of its bounded waits had given up, before it issues any
                             copy or product, so the step ends with NNP_ERR_TIMEOUT */
  int32_t model;          /* nnp_model (0 = ANI-2x, the zero-initialised default) */
  int32_t single_cta;     /* 1: the first layer's tensor-core products on single CTAs
                             (128-row tiles), the path taken when the device cannot hold
                             CTA pairs; 0 = pairs where possible (default) */
  int32_t reserved[2];    /* must be zero */
} nnp_params;

/* Number of FP32 parameters of one ANI-2x ensemble member (1,713,223). */
int64_t nnp_weights_per_model(void);

/* Number of features per atom of ANI-2x (1008). */
int32_t nnp_num_features(void);

/* The same for a given nnp_model (ANI-1x: 326,660 parameters, 384 features);
 * -1 for an unknown model. */
int64_t nnp_weights_per_model_of(int32_t model);
int32_t nnp_num_features_of(int32_t model);

/*
 * Create a handle for one molecule / NNP region of n_atoms atoms with atomic
 * numbers Z (HOST pointer, copied).  Equivalent to nnp_create_batch with one
 * molecule.  Returns NNP_ERR_SPECIES, NNP_ERR_CHARGE, NNP_ERR_ARG or
 * NNP_ERR_ALLOC synchronously; *out is set only on NNP_OK.  Allocates device
 * memory on the current CUDA device and synchronises it.
 */
nnp_status nnp_create(const int32_t* Z, int32_t n_atoms, const nnp_params* params,
                      nnp_handle* out);

/*
 * Create a handle for a batch of n_mols independent molecules (or MD
 * replicas).  Z: HOST [N] atomic numbers, molecule-contiguous; mol_offsets:
 * HOST [n_mols + 1], non-decreasing, mol_offsets[0] = 0, N = mol_offsets[n_mols].
 * Atoms interact only within their molecule.  With a periodic box every
 * molecule uses the same box.
 */
nnp_status nnp_create_batch(const int32_t* Z, const int32_t* mol_offsets, int32_t n_mols,
                            const nnp_params* params, nnp_handle* out);

/*
 * One energy + force evaluation, enqueued on `stream` (a cudaStream_t, may be
 * 0 for the legacy default stream).
 *   positions_dev: DEVICE FP32 [N][3], Angstrom, in the atom order given at
 *                  create time; read only.
 *   energy_out_dev: DEVICE FP64 [n_mols]; written.
 *   forces_out_dev: DEVICE FP64 [N][3] or NULL (energy only); written.
 * The caller owns the three buffers.  No allocation, no host synchronisation.
 * Device-side conditions (capacity overflow, non-finite positions, a bounded
 * wait that gave up) are recorded in a status word read by nnp_get_status;
 * the outputs of such a step are unspecified.  Returns NNP_ERR_ARG or
 * NNP_ERR_CUDA synchronously.
 */
nnp_status nnp_compute(nnp_handle h, const float* positions_dev, double* energy_out_dev,
                       double* forces_out_dev, void* stream);

/*
 * Same as nnp_compute with HOST buffers (pinned or pageable): copies the
 * positions in, evaluates, copies energies and forces out, and synchronises
 * `stream` before returning.  forces_out_host may be NULL.
 */
nnp_status nnp_compute_host(nnp_handle h, const float* positions_host, double* energy_out_host,
                            double* forces_out_host, void* stream);

/* Synchronises the handle's last stream and returns (then clears) the
 * device-side status: NNP_ERR_TIMEOUT if a bounded wait gave up, else
 * NNP_ERR_NONFINITE if a position was not finite, else NNP_ERR_CAPACITY if a
 * neighbour list overflowed (entries beyond the capacity are dropped, never
 * written), else NNP_OK. */
nnp_status nnp_get_status(nnp_handle h);

/* Text of the last error on this handle (static storage owned by the handle;
 * "" if none).  With h == NULL: the last error of a failed create. */
const char* nnp_last_error(nnp_handle h);

/* Free everything the handle owns.  Synchronises the device.  NULL is a no-op. */
void nnp_destroy(nnp_handle h);

/* ---- inspection (diagnostics and parity tests) ------------------------------
 * These read the intermediate results of the LAST nnp_compute on the handle,
 * in the caller's atom order, into caller-owned DEVICE buffers, enqueued on
 * `stream`.  Call after nnp_compute on the same stream. */

/* Neighbour capacities in use (radial, angular). */
nnp_status nnp_get_capacity(nnp_handle h, int32_t* max_radial, int32_t* max_angular);

/* kind 0: radial (r < 5.1 A) neighbours, kind 1: angular (r < 3.5 A).
 * counts_dev: DEVICE int32 [N]; lists_dev: DEVICE int32 [N][cap] (cap >= the
 * handle's capacity for that kind); entries [i][0..counts[i]) are the caller
 * indices of atom i's neighbours, ascending in the handle's internal order
 * (not sorted by caller index); the rest is -1. */
nnp_status nnp_get_neighbors(nnp_handle h, int32_t kind, int32_t* counts_dev, int32_t* lists_dev,
                             int32_t cap, void* stream);

/* Features as the networks consumed them, widened to FP32: DEVICE [N][F], F =
 * nnp_num_features_of(the handle's model). */
nnp_status nnp_get_features(nnp_handle h, float* features_dev, void* stream);

/* Per-atom ensemble-mean energies: DEVICE FP64 [N]. */
nnp_status nnp_get_atomic_energies(nnp_handle h, double* energies_dev, void* stream);

/* ---- measurement -------------------------------------------------------------- */

/* Stages of one evaluation, in launch order.  Fused kernels report in the
 * slot of their first stage: with 16-bit networks, layers 2 and 3 forward,
 * the output layer and (with forces) layers 3 and 2 reverse run in one kernel
 * and report in NNP_STAGE_L2_FWD. */
typedef enum {
  NNP_STAGE_NEIGHBORS = 0, /* position gather + neighbour lists */
  NNP_STAGE_FEATURES = 1,  /* radial + angular features */
  NNP_STAGE_L1_FWD = 2,    /* first layer, all elements and networks */
  NNP_STAGE_L2_FWD = 3,
  NNP_STAGE_L3_FWD = 4,    /* third layer + output layer (energies, start of reverse pass) */
  NNP_STAGE_ENERGY = 5,    /* ensemble mean, FP64 per-molecule sums */
  NNP_STAGE_L3_REV = 6,
  NNP_STAGE_L2_REV = 7,
  NNP_STAGE_L1_REV = 8,    /* dE/dG */
  NNP_STAGE_ADJOINT = 9,   /* featurizer reverse pass, FP64 force accumulation */
  NNP_NUM_STAGES = 10
} nnp_stage;

/* nnp_compute with direct launches and a CUDA event after each stage; waits
 * for the step and writes the stage durations in milliseconds to the HOST
 * array stage_ms[n_stages >= NNP_NUM_STAGES] (stages not run read 0). */
nnp_status nnp_compute_timed(nnp_handle h, const float* positions_dev, double* energy_out_dev,
                             double* forces_out_dev, void* stream, float* stage_ms,
                             int32_t n_stages);

/* Number of kernels one nnp_compute launches (with or without forces). */
int32_t nnp_kernels_per_step(nnp_handle h, int32_t with_forces);

/* Autotuner: times candidate schedules on the given DEVICE positions (as for
 * nnp_compute) and keeps the fastest: atoms (warps) per CTA of the featurizer
 * {2, 4, 8}; warps per CTA {2, 4}, centres per work item and force
 * accumulation (FP64 in shared memory per molecule, or FP64 atomics in global
 * memory) of the featurizer's reverse pass; the N tile {256, 128} of the first
 * layer's tensor-core products.  Synchronises `stream`, allocates and frees
 * scratch for the outputs, and drops a captured graph (captured again on next
 * use).  chosen: HOST int32[5] or NULL, receives (featurizer warps, reverse
 * warps, reverse centres per item, first-layer N tile, shared accumulators). */
nnp_status nnp_autotune(nnp_handle h, const float* positions_dev, void* stream, int32_t* chosen);

/* Applies a schedule that nnp_autotune chose earlier (same five values, same
 * order: featurizer warps per CTA in {2, 4, 8}; reverse warps per CTA in
 * {2, 4}; reverse centres per work item, a multiple of those warps up to 64;
 * first-layer N tile in {128, 256}, ignored for FP32; shared accumulators 0
 * or 1) without timing anything.  schedule: HOST int32[5].  Drops a captured
 * graph.  NNP_ERR_ARG for a null pointer or a value out of range (nothing
 * changes then); NNP_ERR_CUDA if a buffer could not be rebuilt. */
nnp_status nnp_set_schedule(nnp_handle h, const int32_t* schedule);

/* ---- allocation-free entry point -----------------------------------------------
 * The paper has no counterpart: this serves callers that cannot let a library
 * allocate device memory -- an MD engine capturing its whole time step into a
 * CUDA graph (cudaMalloc cannot be captured and synchronises the device), or a
 * host framework that owns the device memory budget and forbids raw
 * cudaMalloc.  It needs no handle and allocates nothing.
 *
 * Features of ONE non-periodic molecule, the same quantities nnp_get_features
 * returns after nnp_compute:
 *   Z_dev:            DEVICE int32 [n_atoms] atomic numbers
 *   positions_dev:    DEVICE FP32 [n_atoms][3], Angstrom
 *   features_out_dev: DEVICE FP32 [n_atoms][1008], written (caller order)
 * n_atoms > NNP_STATIC_MAX_ATOMS returns NNP_ERR_TOO_LARGE; nothing is enqueued.
 * An atomic number outside {1,6,7,8,9,16,17} or a non-finite position makes
 * every output feature NaN (there is no handle to carry a status).
 * Intermediates live in one fixed scratch array of about 1.6 MB in device global
 * memory that every GPU loading the library holds until the process exits;
 * all calls on a device share it and it keeps the last call's contents, so
 * calls that overlap on the GPU race: serialise them (one stream, or events).
 * The first call on each device looks up the array's address (with that
 * device current); make that first call before any stream capture.  The
 * stream must belong to the current device (the scratch array is per device).
 * Returns NNP_ERR_ARG for null buffers or a stream of another device,
 * NNP_ERR_CUDA if a launch failed. */
#define NNP_STATIC_MAX_ATOMS 256
nnp_status nnp_features_static(const int32_t* Z_dev, const float* positions_dev, int32_t n_atoms,
                               float* features_out_dev, void* stream);

/* ---- NNP-MM coupling term ---------------------------------------------------------
 * The coupling term of the hybrid potential (Eq. 4, the mechanical-embedding
 * scheme of Sec. 2): Coulomb plus Lennard-Jones between every NNP atom i and
 * every MM atom j,
 *   V = sum_i sum_j  coulomb_k q_i q_j / r_ij
 *                  + 4 eps_ij ((sigma_ij / r_ij)^12 - (sigma_ij / r_ij)^6),
 *   sigma_ij = (sigma_i + sigma_j) / 2,  eps_ij = sqrt(eps_i eps_j)  (Lorentz-Berthelot),
 * with no cutoff and no periodic images, as the equation is written (the MM
 * engine treats the MM region's own long-range electrostatics).  coulomb_k is
 * 1 / (4 pi eps0) in the caller's units (332.0637133 kcal/mol A / e^2 for
 * positions in A, charges in e and eps in kcal/mol).  It needs no handle and
 * allocates nothing; it is asynchronous on `stream`.
 *   nnp_positions_dev, mm_positions_dev: DEVICE FP32 [n][3];
 *   *_charges_dev, *_sigma_dev, *_epsilon_dev: DEVICE FP32 [n] (eps >= 0);
 *   energy_dev: DEVICE FP64 scalar, the term's energy is ADDED to it;
 *   nnp_forces_dev [n_nnp][3], mm_forces_dev [n_mm][3]: DEVICE FP64, the forces
 *     -dV/dx are ADDED (so the NNP forces of nnp_compute can be passed as is).
 * Pair arithmetic is FP32, sums FP64 across warps; results differ between calls
 * only by the order of FP64 additions across CTAs.  Returns NNP_ERR_ARG for
 * negative counts or null buffers, NNP_ERR_TOO_LARGE for more than
 * NNP_COUPLING_MAX_NNP NNP atoms (they are staged in shared memory), NNP_OK
 * without work when a count is 0, NNP_ERR_CUDA if the launch failed.  An NNP
 * atom and an MM atom at the same position make the outputs non-finite. */
#define NNP_COUPLING_MAX_NNP 512
nnp_status nnp_mm_coupling(const float* nnp_positions_dev, const float* nnp_charges_dev,
                           const float* nnp_sigma_dev, const float* nnp_epsilon_dev, int32_t n_nnp,
                           const float* mm_positions_dev, const float* mm_charges_dev,
                           const float* mm_sigma_dev, const float* mm_epsilon_dev, int32_t n_mm,
                           double coulomb_k, double* energy_dev, double* nnp_forces_dev,
                           double* mm_forces_dev, void* stream);

/* ---- replica MD loop -----------------------------------------------------------------
 * Molecular dynamics of every atom of a handle (its molecules are independent
 * replicas) with the NNP term and, optionally, the NNP-MM coupling term
 * (nnp_mm_coupling) of one fixed MM environment that every replica sees.  The
 * paper keeps the MD step on the GPU (Sec. 2 "Optimization") and names the
 * serial execution of the NNP and MM force terms as what is left to gain
 * (Sec. 3, after the MD speed table): here each step is one CUDA graph replay
 * and the coupling term can run on a second stream beside the NNP term.
 *   velocity Verlet: v += dt/2 F/m; x += dt v; F = F(x); v += dt/2 F/m
 *   Langevin BAOAB:  v += dt/2 F/m; x += dt/2 v; v = c1 v + c2 sqrt(kT/m) xi;
 *                    x += dt/2 v; F = F(x); v += dt/2 F/m,
 *                    c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2), xi ~ N(0, 1)
 * Positions and velocities are FP64 in the caller's buffers (the NNP takes the
 * positions rounded to FP32); forces are the FP64 sums of nnp_compute and the
 * coupling term.  Units are the caller's, consistent with the network's
 * energy unit (forces per Angstrom): dt, masses, kT. */
typedef struct nnp_md* nnp_md_handle;

typedef enum { NNP_MD_VERLET = 0, NNP_MD_BAOAB = 1 } nnp_md_integrator;

typedef struct {
  int32_t integrator;          /* nnp_md_integrator */
  double dt;                   /* time step, > 0 */
  double gamma;                /* friction coefficient (BAOAB), >= 0 */
  double kT;                   /* thermal energy (BAOAB), >= 0 */
  const double* masses;        /* HOST [N], caller order, > 0; copied */
  int32_t n_mm;                /* MM atoms of the environment; 0 = no coupling term */
  const float* mm_positions_dev;  /* DEVICE [n_mm][3] (held, not copied; fixed atoms) */
  const float* mm_charges_dev;    /* DEVICE [n_mm] */
  const float* mm_sigma_dev;      /* DEVICE [n_mm] */
  const float* mm_epsilon_dev;    /* DEVICE [n_mm] */
  const float* nnp_charges_dev;   /* DEVICE [N] coupling parameters of the handle's atoms */
  const float* nnp_sigma_dev;     /* DEVICE [N] */
  const float* nnp_epsilon_dev;   /* DEVICE [N] */
  double coulomb_k;               /* 1 / (4 pi eps0) in the caller's units */
  int32_t concurrent;          /* 1: the coupling term on a second stream beside the NNP term */
  int32_t reserved[8];         /* must be zero */
} nnp_md_params;

/* Create the loop for handle nnp (which must outlive it; its own graph
 * setting is not used: the loop captures the NNP kernels into its step
 * graph).  NNP_ERR_ARG for bad parameters, NNP_ERR_TOO_LARGE if a replica
 * has more than NNP_COUPLING_MAX_NNP atoms with a coupling term.  Allocates
 * device memory and synchronises the device. */
nnp_status nnp_md_create(nnp_handle nnp, const nnp_md_params* params, nnp_md_handle* out);

/* n_steps steps from the state in x_dev / v_dev (DEVICE FP64 [N][3], caller
 * order, updated in place), enqueued on `stream`: the forces at the starting
 * positions, then one graph replay per step.
 *   noise_dev:  DEVICE FP64 [n_steps][N][3] standard normal draws (BAOAB; row
 *               k is step k's; ignored by Verlet, may be NULL then)
 *   energy_dev: DEVICE FP64 [n_steps][n_mols] or NULL: the potential energy
 *               (NNP + coupling) of each replica after each step
 * No allocation and no host synchronisation after the first call with a
 * given set of buffers (which captures the step graph).  Device-side
 * conditions are reported by nnp_get_status on the NNP handle. */
nnp_status nnp_md_run(nnp_md_handle md, double* x_dev, double* v_dev, int32_t n_steps,
                      const double* noise_dev, double* energy_dev, void* stream);

const char* nnp_md_last_error(nnp_md_handle md);

/* Free the loop's buffers (not the NNP handle).  Synchronises the device. */
void nnp_md_destroy(nnp_md_handle md);

#ifdef __cplusplus
}
#endif

#endif /* NNP_H_ */
