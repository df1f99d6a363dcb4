// md.cu -- the replica MD loop around the NNP term: velocity Verlet or
// Langevin (BAOAB) dynamics of every atom of a handle (its molecules are the
// replicas), each step one CUDA graph replay of
//   first half  (FP64): B  v += dt/2 F/m,  then  A  x += dt v  (Verlet), or
//                       A  x += dt/2 v,  O  v = c1 v + c2 sqrt(kT/m) xi,
//                       A  x += dt/2 v  (BAOAB); x rounded to FP32 for the NNP;
//   forces:             the NNP term (the handle's kernels) and, optionally,
//                       the NNP-MM coupling term of one fixed MM environment
//                       for every replica, on a second stream beside it;
//   second half (FP64): B  v += dt/2 (F_NNP + F_coupling)/m, and the potential
//                       energy of every replica recorded for the step.
// The paper keeps the whole MD step on the GPU (Sec. 2 "Optimization") and
// names the serial execution of the NNP and MM force terms as what is left
// to gain (Sec. 3, after the MD speed table); here the coupling term runs on
// its own stream concurrently with the NNP term.  The step index that selects
// the noise row and the energy row lives in device memory, so one captured
// graph serves every step.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/nnp.h"
#include "nnp_internal.cuh"

struct nnp_md {
  nnp_handle nnp = nullptr;
  int n = 0, n_mols = 0;
  std::vector<int> mol_off;
  int integrator = 0;
  double dt = 0.0, c1 = 1.0, c2 = 0.0, kT = 0.0;
  double* d_minv = nullptr;  // [N] 1 / m
  float* d_x32 = nullptr;    // [N][3] positions as the NNP takes them
  double* d_F = nullptr;     // [N][3] NNP forces
  double* d_E = nullptr;     // [n_mols] NNP energies
  double* d_Fc = nullptr;    // [N][3] coupling forces on the NNP atoms
  double* d_Ec = nullptr;    // [n_mols] coupling energies
  double* d_Fmm = nullptr;   // [n_mm][3] coupling forces on the (fixed) MM atoms, not used
  int* d_step = nullptr;
  // coupling term (device pointers held, not copied)
  int n_mm = 0;
  const float *mm_x = nullptr, *mm_q = nullptr, *mm_s = nullptr, *mm_e = nullptr;
  const float *nq = nullptr, *ns = nullptr, *ne = nullptr;
  double ke = 0.0;
  int concurrent = 0;
  cudaStream_t cap = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const double* g_noise = nullptr;
  double *g_x = nullptr, *g_v = nullptr, *g_energy = nullptr;
  std::string err;
};

namespace {

constexpr int kMdThreads = 128;

// First half of a step, one thread per atom; also zeroes the coupling
// accumulators the step's force evaluation adds into.
__global__ void k_md_first(int n, int n_mols, int baoab, double dt, double c1, double c2, double kT,
                           const double* __restrict__ minv, double* __restrict__ x,
                           double* __restrict__ v, const double* __restrict__ F,
                           double* __restrict__ Fc, double* __restrict__ Ec,
                           const double* __restrict__ noise, const int* __restrict__ step,
                           float* __restrict__ x32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_mols && Ec) Ec[i] = 0.0;
  if (i >= n) return;
  const double mi = minv[i];
  const double* xi_row = baoab ? noise + (size_t)(*step) * n * 3 : nullptr;
  const double sigma = baoab ? c2 * sqrt(kT * mi) : 0.0;
  for (int d = 0; d < 3; ++d) {
    const size_t k = 3 * (size_t)i + d;
    const double f = F[k] + (Fc ? Fc[k] : 0.0);
    double vk = v[k] + 0.5 * dt * f * mi;
    double xk = x[k];
    if (baoab) {
      xk += 0.5 * dt * vk;
      vk = c1 * vk + sigma * xi_row[k];
      xk += 0.5 * dt * vk;
    } else {
      xk += dt * vk;
    }
    v[k] = vk;
    x[k] = xk;
    x32[k] = (float)xk;
    if (Fc) Fc[k] = 0.0;
  }
}

// Second half: the closing half kick with the new forces.
__global__ void k_md_second(int n, double dt, const double* __restrict__ minv, double* __restrict__ v,
                            const double* __restrict__ F, const double* __restrict__ Fc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double h = 0.5 * dt * minv[i];
  for (int d = 0; d < 3; ++d) {
    const size_t k = 3 * (size_t)i + d;
    v[k] += h * (F[k] + (Fc ? Fc[k] : 0.0));
  }
}

// The step's potential energies (NNP + coupling) per replica into row *step
// of the output, then the step index advances (one CTA: every thread has read
// the index before thread 0 writes it).
__global__ void k_md_record(int n_mols, const double* __restrict__ E, const double* __restrict__ Ec,
                            double* __restrict__ out, int* __restrict__ step) {
  const int s = *step;
  if (out)
    for (int r = threadIdx.x; r < n_mols; r += blockDim.x)
      out[(size_t)s * n_mols + r] = E[r] + (Ec ? Ec[r] : 0.0);
  __syncthreads();
  if (threadIdx.x == 0) *step = s + 1;
}

// Positions to FP32 and the coupling accumulators to zero (the force
// evaluation at the start of a run).
__global__ void k_md_start(int n, int n_mols, const double* __restrict__ x, float* __restrict__ x32,
                           double* __restrict__ Fc, double* __restrict__ Ec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_mols && Ec) Ec[i] = 0.0;
  if (i >= 3 * n) return;
  x32[i] = (float)x[i];
  if (Fc) Fc[i] = 0.0;
}

nnp_status md_fail(nnp_md* md, nnp_status st, const std::string& msg) {
  if (md) md->err = msg;
  return st;
}

// A failed call's error is also taken off the thread's last-error state, so
// that it does not surface in a later, unrelated call.
#define MDCK(call)                                                                           \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      cudaGetLastError();                                                                    \
      return md_fail(md, e_ == cudaErrorMemoryAllocation ? NNP_ERR_ALLOC : NNP_ERR_CUDA,     \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    }                                                                                        \
  } while (0)

// The forces at md->d_x32: the NNP term on s, the coupling term on the side
// stream (concurrent) or after it on s.
nnp_status enqueue_forces(nnp_md* md, cudaStream_t s) {
  const bool cpl = md->n_mm > 0;
  cudaStream_t sc = s;
  if (cpl && md->concurrent) {
    MDCK(cudaEventRecord(md->ev_fork, s));
    MDCK(cudaStreamWaitEvent(md->side, md->ev_fork, 0));
    sc = md->side;
  }
  if (cpl) {
    for (int r = 0; r < md->n_mols; ++r) {
      const int a0 = md->mol_off[r], na = md->mol_off[r + 1] - a0;
      const nnp_status st = nnp_mm_coupling(md->d_x32 + 3 * (size_t)a0, md->nq + a0, md->ns + a0,
                                            md->ne + a0, na, md->mm_x, md->mm_q, md->mm_s, md->mm_e,
                                            md->n_mm, md->ke, md->d_Ec + r, md->d_Fc + 3 * (size_t)a0,
                                            md->d_Fmm, sc);
      if (st != NNP_OK) return md_fail(md, st, "coupling term launch failed");
    }
  }
  if (nnp::enqueue_nnp(md->nnp, md->d_x32, md->d_E, md->d_F, s) < 0)
    return md_fail(md, NNP_ERR_CUDA, "NNP term launch failed");
  if (cpl && md->concurrent) {
    MDCK(cudaEventRecord(md->ev_join, md->side));
    MDCK(cudaStreamWaitEvent(s, md->ev_join, 0));
  }
  return NNP_OK;
}

nnp_status enqueue_md_step(nnp_md* md, double* x, double* v, const double* noise, double* energy,
                           cudaStream_t s) {
  const int blocks = (md->n + kMdThreads - 1) / kMdThreads;
  const int blocks_first = (std::max(md->n, md->n_mols) + kMdThreads - 1) / kMdThreads;
  const bool cpl = md->n_mm > 0;
  k_md_first<<<blocks_first, kMdThreads, 0, s>>>(md->n, md->n_mols, md->integrator, md->dt, md->c1,
                                                 md->c2, md->kT, md->d_minv, x, v, md->d_F,
                                                 cpl ? md->d_Fc : nullptr, cpl ? md->d_Ec : nullptr,
                                                 noise, md->d_step, md->d_x32);
  const nnp_status st = enqueue_forces(md, s);
  if (st != NNP_OK) return st;
  k_md_second<<<blocks, kMdThreads, 0, s>>>(md->n, md->dt, md->d_minv, v, md->d_F,
                                           cpl ? md->d_Fc : nullptr);
  k_md_record<<<1, 256, 0, s>>>(md->n_mols, md->d_E, cpl ? md->d_Ec : nullptr, energy, md->d_step);
  return NNP_OK;
}

template <typename T>
cudaError_t md_alloc(T** p, size_t count) {
  *p = nullptr;
  return cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
}

}  // namespace

extern "C" {

void nnp_md_destroy(nnp_md_handle md) {
  if (!md) return;
  cudaDeviceSynchronize();
  if (md->gexec) cudaGraphExecDestroy(md->gexec);
  if (md->cap) cudaStreamDestroy(md->cap);
  if (md->side) cudaStreamDestroy(md->side);
  if (md->ev_fork) cudaEventDestroy(md->ev_fork);
  if (md->ev_join) cudaEventDestroy(md->ev_join);
  for (void* p : {(void*)md->d_minv, (void*)md->d_x32, (void*)md->d_F, (void*)md->d_E, (void*)md->d_Fc,
                  (void*)md->d_Ec, (void*)md->d_Fmm, (void*)md->d_step})
    if (p) cudaFree(p);
  delete md;
}

nnp_status nnp_md_create(nnp_handle nnp, const nnp_md_params* p, nnp_md_handle* out) {
  nnp_md* md = nullptr;
  if (!nnp || !p || !out) return NNP_ERR_ARG;
  *out = nullptr;
  if (p->integrator != NNP_MD_VERLET && p->integrator != NNP_MD_BAOAB) return NNP_ERR_ARG;
  if (!(p->dt > 0.0) || p->gamma < 0.0 || p->kT < 0.0 || !p->masses || p->n_mm < 0) return NNP_ERR_ARG;
  for (int r = 0; r < 8; ++r)
    if (p->reserved[r] != 0) return NNP_ERR_ARG;
  if (p->n_mm > 0 && (!p->mm_positions_dev || !p->mm_charges_dev || !p->mm_sigma_dev ||
                      !p->mm_epsilon_dev || !p->nnp_charges_dev || !p->nnp_sigma_dev ||
                      !p->nnp_epsilon_dev))
    return NNP_ERR_ARG;
  md = new nnp_md();
  md->nnp = nnp;
  nnp::handle_shape(nnp, &md->n, &md->n_mols, md->mol_off);
  for (int r = 0; r < md->n_mols; ++r)
    if (p->n_mm > 0 && md->mol_off[r + 1] - md->mol_off[r] > NNP_COUPLING_MAX_NNP) {
      delete md;
      return NNP_ERR_TOO_LARGE;
    }
  for (int i = 0; i < md->n; ++i)
    if (!(p->masses[i] > 0.0)) {
      delete md;
      return NNP_ERR_ARG;
    }
  struct Guard {
    nnp_md*& md;
    bool ok = false;
    ~Guard() {
      if (!ok && md) nnp_md_destroy(md);
    }
  } guard{md};
  md->integrator = p->integrator;
  md->dt = p->dt;
  md->kT = p->kT;
  md->c1 = std::exp(-p->gamma * p->dt);
  md->c2 = std::sqrt(std::max(0.0, 1.0 - md->c1 * md->c1));
  md->n_mm = p->n_mm;
  md->mm_x = p->mm_positions_dev;
  md->mm_q = p->mm_charges_dev;
  md->mm_s = p->mm_sigma_dev;
  md->mm_e = p->mm_epsilon_dev;
  md->nq = p->nnp_charges_dev;
  md->ns = p->nnp_sigma_dev;
  md->ne = p->nnp_epsilon_dev;
  md->ke = p->coulomb_k;
  md->concurrent = p->concurrent;
  const int N = md->n;
  std::vector<double> minv(N);
  for (int i = 0; i < N; ++i) minv[i] = 1.0 / p->masses[i];
  MDCK(md_alloc(&md->d_minv, N));
  MDCK(cudaMemcpy(md->d_minv, minv.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  MDCK(md_alloc(&md->d_x32, 3 * (size_t)N));
  MDCK(md_alloc(&md->d_F, 3 * (size_t)N));
  MDCK(md_alloc(&md->d_E, md->n_mols));
  MDCK(md_alloc(&md->d_Fc, 3 * (size_t)N));
  MDCK(md_alloc(&md->d_Ec, md->n_mols));
  MDCK(md_alloc(&md->d_Fmm, 3 * (size_t)std::max(md->n_mm, 1)));
  MDCK(cudaMemset(md->d_Fmm, 0, sizeof(double) * 3 * std::max(md->n_mm, 1)));
  MDCK(md_alloc(&md->d_step, 1));
  MDCK(cudaStreamCreateWithFlags(&md->cap, cudaStreamNonBlocking));
  MDCK(cudaStreamCreateWithFlags(&md->side, cudaStreamNonBlocking));
  MDCK(cudaEventCreateWithFlags(&md->ev_fork, cudaEventDisableTiming));
  MDCK(cudaEventCreateWithFlags(&md->ev_join, cudaEventDisableTiming));
  MDCK(cudaDeviceSynchronize());
  guard.ok = true;
  *out = md;
  return NNP_OK;
}

nnp_status nnp_md_run(nnp_md_handle md, double* x_dev, double* v_dev, int32_t n_steps,
                      const double* noise_dev, double* energy_dev, void* stream) {
  if (!md || n_steps < 0 || !x_dev || !v_dev) return NNP_ERR_ARG;
  cudaGetLastError();  // a stale error of the caller's must not be taken for one of these launches
  if (md->integrator == NNP_MD_BAOAB && n_steps > 0 && !noise_dev)
    return md_fail(md, NNP_ERR_ARG, "BAOAB needs the normal draws");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  nnp::set_last_stream(md->nnp, s);
  const bool cpl = md->n_mm > 0;
  // forces at the starting positions, and the step index to 0
  const int nb = (std::max(3 * md->n, md->n_mols) + kMdThreads - 1) / kMdThreads;
  k_md_start<<<nb, kMdThreads, 0, s>>>(md->n, md->n_mols, x_dev, md->d_x32, cpl ? md->d_Fc : nullptr,
                                       cpl ? md->d_Ec : nullptr);
  MDCK(cudaMemsetAsync(md->d_step, 0, sizeof(int), s));
  nnp_status st = enqueue_forces(md, s);
  if (st != NNP_OK) return st;
  MDCK(cudaGetLastError());
  if (n_steps == 0) return NNP_OK;
  // one graph per set of buffers: the step's kernels and both force terms
  if (!md->gexec || md->g_x != x_dev || md->g_v != v_dev || md->g_noise != noise_dev ||
      md->g_energy != energy_dev) {
    if (md->gexec) {
      cudaGraphExecDestroy(md->gexec);
      md->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    MDCK(cudaStreamBeginCapture(md->cap, cudaStreamCaptureModeThreadLocal));
    st = enqueue_md_step(md, x_dev, v_dev, noise_dev, energy_dev, md->cap);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ce = cudaStreamEndCapture(md->cap, &graph);
    if (st != NNP_OK || le != cudaSuccess || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return st != NNP_OK ? st
                          : md_fail(md, NNP_ERR_CUDA, std::string("MD step capture: ") +
                                                          cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    const cudaError_t ie = cudaGraphInstantiate(&md->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      md->gexec = nullptr;
      return md_fail(md, NNP_ERR_CUDA, std::string("MD step instantiate: ") + cudaGetErrorString(ie));
    }
    md->g_x = x_dev;
    md->g_v = v_dev;
    md->g_noise = noise_dev;
    md->g_energy = energy_dev;
  }
  for (int k = 0; k < n_steps; ++k) MDCK(cudaGraphLaunch(md->gexec, s));
  return NNP_OK;
}

const char* nnp_md_last_error(nnp_md_handle md) { return md ? md->err.c_str() : ""; }

}  // extern "C"
