// aev.cu -- neighbour lists, the ANI featurizer and its reverse pass.
//
// Neighbour search: one warp per centre atom scans its molecule (or periodic
// region) 32 candidates at a time; a ballot and a prefix popcount compact the
// accepted candidates in ascending internal index, so every list is sorted
// and therefore grouped by element.  The cutoff test is FP32 with an FP64
// recheck of the exact squared distance inside a 1e-4 relative guard band,
// which makes the pair sets identical to an FP64 evaluation.
//
// Featurizer (the modified Behler-Parrinello functions the paper names in
// Sec. 1; Sec. 2 "Optimization" describes the custom CUDA featurizer): one
// warp per centre.  Radial terms: lanes = 16 shifts x 2 neighbours, summed
// into a per-warp shared-memory row (each lane owns one column: no atomics).
// Angular terms, two phases per 32 neighbour pairs: (1) lane per pair
// computes the 4 angle factors, 8 distance factors and its species-pair block;
// (2) lane per feature (8 x 4) walks the 32 pairs and accumulates
// R_a * A_z into the block in registers, flushing on a block change.
//
// Reverse pass: one warp per centre, lane per neighbour (radial) and lane per
// pair (angular); per-neighbour gradients gather in shared memory, then go to
// a per-warp FP64 accumulator of the molecule (or FP64 global atomics for
// large regions); each CTA adds its molecule totals to the forces with FP64
// atomics.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

constexpr float kPi = 3.14159265358979323846f;

__device__ __forceinline__ float3 min_image(float3 d, const AevConst& c) {
  if (c.periodic) {
    d.x -= c.box[0] * rintf(d.x / c.box[0]);
    d.y -= c.box[1] * rintf(d.y / c.box[1]);
    d.z -= c.box[2] * rintf(d.z / c.box[2]);
  }
  return d;
}

__device__ __forceinline__ float3 disp(float4 xi, float4 xj, const AevConst& c) {
  return min_image(make_float3(xj.x - xi.x, xj.y - xi.y, xj.z - xi.z), c);
}

// Exact FP64 squared distance of two FP32 positions, every operation rounded
// on its own (no contraction), minimum image d - L floor(d / L + 1/2).
__device__ double exact_d2(float4 xi, float4 xj, const AevConst& c) {
  double d[3] = {__dsub_rn((double)xj.x, (double)xi.x), __dsub_rn((double)xj.y, (double)xi.y),
                 __dsub_rn((double)xj.z, (double)xi.z)};
  if (c.periodic) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double L = c.boxd[k];
      const double n = floor(__dadd_rn(__ddiv_rn(d[k], L), 0.5));
      d[k] = __dsub_rn(d[k], __dmul_rn(L, n));
    }
  }
  double s = __dmul_rn(d[0], d[0]);
  s = __dadd_rn(s, __dmul_rn(d[1], d[1]));
  s = __dadd_rn(s, __dmul_rn(d[2], d[2]));
  return s;
}

__global__ void k_neighbors(Geometry g, NeighborLists nl, AevConst c, unsigned* status) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= g.n_atoms) return;
  const int a0 = g.mol_start[q], a1 = g.mol_end[q];
  const float4 xi = g.pos[q];
  const unsigned lt = (1u << lane) - 1u;
  int nr = 0, na = 0;
  int* lr = nl.nbr_r + (size_t)q * nl.cap_r;
  int* la = nl.nbr_a + (size_t)q * nl.cap_a;
  int* sa = nl.slot_a + (size_t)q * nl.cap_a;
  for (int base = a0; base < a1; base += 32) {
    const int j = base + lane;
    bool inR = false, inA = false;
    if (j < a1 && j != q) {
      const float4 xj = g.pos[j];
      const float3 d = disp(xi, xj, c);
      const float d2 = d.x * d.x + d.y * d.y + d.z * d.z;
      inR = d2 < c.Rcr2;
      inA = d2 < c.Rca2;
      if (fabsf(d2 - c.Rcr2) <= 1e-4f * c.Rcr2) inR = exact_d2(xi, xj, c) < c.Rcr2d;
      if (fabsf(d2 - c.Rca2) <= 1e-4f * c.Rca2) inA = exact_d2(xi, xj, c) < c.Rca2d;
      inA = inA && inR;
    }
    const unsigned mR = __ballot_sync(0xffffffffu, inR);
    const unsigned mA = __ballot_sync(0xffffffffu, inA);
    if (inR) {
      const int slot = nr + __popc(mR & lt);
      if (slot < nl.cap_r) lr[slot] = j;
      if (inA) {
        const int sl = na + __popc(mA & lt);
        if (sl < nl.cap_a) {
          la[sl] = j;
          sa[sl] = slot;
        }
      }
    }
    nr += __popc(mR);
    na += __popc(mA);
  }
  if (lane == 0) {
    nl.cnt_r[q] = nr;
    nl.cnt_a[q] = na;
    if (nr > nl.cap_r) atomicOr(status, kStatCapRadial);
    if (na > nl.cap_a) atomicOr(status, kStatCapAngular);
  }
}

// Row j and column k of the P-th pair (j < k) of n items, pairs ordered
// row-major over the strict upper triangle.
__device__ __forceinline__ void decode_pair(int P, int n, int& j, int& k) {
  const float b = (float)(2 * n - 1);
  int jj = (int)((b - sqrtf(fmaxf(b * b - 8.f * (float)P, 0.f))) * 0.5f);
  jj = max(0, min(jj, n - 2));
  // start of row r: r (2n - r - 1) / 2
  while (jj > 0 && (jj * (2 * n - jj - 1)) / 2 > P) --jj;
  while (jj + 1 <= n - 2 && ((jj + 1) * (2 * n - jj - 2)) / 2 <= P) ++jj;
  j = jj;
  k = P - (jj * (2 * n - jj - 1)) / 2 + jj + 1;
}

template <typename T> __device__ __forceinline__ T cvt_out(float v);
template <> __device__ __forceinline__ float cvt_out<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half cvt_out<__half>(float v) { return __float2half_rn(v); }

// Per-warp shared memory of the forward kernel (floats).
__host__ __device__ constexpr int aev_fwd_warp_floats(int cap_a) {
  return kAngular + 2 * kRadial + 32 * 13 + cap_a * 6;
}

template <typename TOut>
__global__ void k_aev(Geometry g, NeighborLists nl, AevConst c, const int* __restrict__ row_of_int,
                      TOut* __restrict__ out) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + warp;
  if (q >= g.n_atoms) return;  // warp-uniform; no block-level barriers below
  float* Gang = smem + (size_t)warp * aev_fwd_warp_floats(nl.cap_a);
  float* R2 = Gang + kAngular;          // [2][112]
  float* buf = R2 + 2 * kRadial;        // [32][13]
  float4* nb = reinterpret_cast<float4*>(buf + 32 * 13);  // [cap_a]  (16-byte aligned: see host)
  float* nfc = reinterpret_cast<float*>(nb + nl.cap_a);    // [cap_a]
  int* nsp = reinterpret_cast<int*>(nfc + nl.cap_a);       // [cap_a]

  for (int f = lane; f < kAngular; f += 32) Gang[f] = 0.f;
  for (int f = lane; f < 2 * kRadial; f += 32) R2[f] = 0.f;
  const float4 xi = g.pos[q];

  // ---- radial: lane = (half, shift) ----
  {
    const int nr = min(nl.cnt_r[q], nl.cap_r);
    const int half = lane >> 4, k = lane & 15;
    const float shf = c.ShfR[k];
    const int* lr = nl.nbr_r + (size_t)q * nl.cap_r;
    float* acc = R2 + half * kRadial;
    __syncwarp();
    for (int t = half; t < nr; t += 2) {
      const int j = lr[t];
      const float3 d = disp(xi, g.pos[j], c);
      const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
      const float fc = 0.5f * cospif(r / c.Rcr) + 0.5f;
      const float x = r - shf;
      acc[g.species[j] * kShfR + k] += 0.25f * expf(-c.EtaR * x * x) * fc;
    }
  }

  // ---- angular ----
  const int na = min(nl.cnt_a[q], nl.cap_a);
  {
    const int* la = nl.nbr_a + (size_t)q * nl.cap_a;
    for (int t = lane; t < na; t += 32) {
      const int j = la[t];
      const float3 d = disp(xi, g.pos[j], c);
      const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
      nb[t] = make_float4(d.x, d.y, d.z, r);
      nfc[t] = 0.5f * cospif(r / c.Rca) + 0.5f;
      nsp[t] = g.species[j];
    }
  }
  __syncwarp();
  const int T = na * (na - 1) / 2;
  const int fa = lane >> 2, fz = lane & 3;
  float acc = 0.f;
  int pcur = -1;
  for (int base = 0; base < T; base += 32) {
    const int P = base + lane;
    float* my = buf + lane * 13;
    if (P < T) {
      int j, k;
      decode_pair(P, na, j, k);
      const float4 rj = nb[j], rk = nb[k];
      const float cost = (rj.x * rk.x + rj.y * rk.y + rj.z * rk.z) / (rj.w * rk.w);
      const float cp = 0.95f * cost;
      const float sp = sqrtf(fmaxf(1.f - cp * cp, 0.f));
      const float fcjk = nfc[j] * nfc[k];
      const float u = 0.5f * (rj.w + rk.w);
#pragma unroll
      for (int a = 0; a < kShfA; ++a) {
        const float x = u - c.ShfA[a];
        my[a] = expf(-c.EtaA * x * x);
      }
#pragma unroll
      for (int z = 0; z < kShfZ; ++z) {
        const float b = fmaxf(0.5f * (1.f + cp * c.cosZ[z] + sp * c.sinZ[z]), 0.f);
        my[kShfA + z] = 2.f * exp2f(c.Zeta * log2f(b)) * fcjk;
      }
      my[12] = __int_as_float(c.pair_index[nsp[j]][nsp[k]]);
    }
    __syncwarp();
    const int cnt = min(32, T - base);
    for (int t = 0; t < cnt; ++t) {
      const float* row = buf + t * 13;
      const int p = __float_as_int(row[12]);
      if (p != pcur) {
        if (pcur >= 0) Gang[pcur * kAngPerBlock + lane] += acc;
        acc = 0.f;
        pcur = p;
      }
      acc = fmaf(row[fa], row[kShfA + fz], acc);
    }
    __syncwarp();
  }
  if (pcur >= 0) Gang[pcur * kAngPerBlock + lane] += acc;
  __syncwarp();

  TOut* dst = out + (size_t)row_of_int[q] * kFeaturesPad;
  for (int f = lane; f < kFeaturesPad; f += 32) {
    float v;
    if (f < kRadial) v = R2[f] + R2[kRadial + f];
    else if (f < kFeatures) v = Gang[f - kRadial];
    else v = 0.f;
    dst[f] = cvt_out<TOut>(v);
  }
}

// ---------------------------------------------------------------------------
// Reverse pass.

constexpr int kGAStride = 33;  // padded row of an angular block (bank spread)

__host__ __device__ constexpr int adj_warp_floats(int cap_r, int cap_a) {
  // gR[112] | gA[28*33] (+pad to 4) | nb float4[cap_a] | nfc, ndfc, nsp, nslot [cap_a] | sg[cap_r*3]
  return ((kRadial + kPairBlocks * kGAStride + 3) / 4) * 4 + cap_a * 4 + cap_a * 4 + cap_r * 3;
}

__device__ __forceinline__ void add_force(double* acc_w, int local, const int* orig, int a_glob,
                                          double* F, float gx, float gy, float gz) {
  if (acc_w) {
    acc_w[3 * local + 0] += (double)gx;
    acc_w[3 * local + 1] += (double)gy;
    acc_w[3 * local + 2] += (double)gz;
  } else {
    const size_t o = 3 * (size_t)orig[a_glob];
    atomicAdd(F + o + 0, -(double)gx);
    atomicAdd(F + o + 1, -(double)gy);
    atomicAdd(F + o + 2, -(double)gz);
  }
}

__global__ void k_aev_adjoint(Geometry g, NeighborLists nl, AevConst c,
                              const int* __restrict__ row_of_int, const float* __restrict__ dG,
                              const int4* __restrict__ work, const int* __restrict__ orig,
                              double* __restrict__ F, int smem_atoms_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 w = work[blockIdx.x];
  const int a0 = w.x, n_mol = w.y, q0 = w.z, q1 = w.w;
  const bool smem_acc = n_mol <= smem_atoms_max;
  double* accm = reinterpret_cast<double*>(smem_raw);  // [nwarps][smem_atoms_max][3]
  float* wbase = reinterpret_cast<float*>(accm + (size_t)nwarps * smem_atoms_max * 3) +
                 (size_t)warp * adj_warp_floats(nl.cap_r, nl.cap_a);
  float* gR = wbase;
  float* gA = gR + kRadial;
  float4* nb = reinterpret_cast<float4*>(wbase + ((kRadial + kPairBlocks * kGAStride + 3) / 4) * 4);
  float* nfc = reinterpret_cast<float*>(nb + nl.cap_a);
  float* ndfc = nfc + nl.cap_a;
  int* nsp = reinterpret_cast<int*>(ndfc + nl.cap_a);
  int* nslot = nsp + nl.cap_a;
  float* sg = reinterpret_cast<float*>(nslot + nl.cap_a);  // [cap_r][3]
  double* acc_w = smem_acc ? accm + (size_t)warp * smem_atoms_max * 3 : nullptr;

  if (smem_acc)
    for (int t = threadIdx.x; t < nwarps * smem_atoms_max * 3; t += blockDim.x) accm[t] = 0.0;
  __syncthreads();

  for (int q = q0 + warp; q < q1; q += nwarps) {
    const float* grow = dG + (size_t)row_of_int[q] * kFeaturesPad;
    for (int f = lane; f < kRadial; f += 32) gR[f] = grow[f];
    for (int f = lane; f < kAngular; f += 32)
      gA[(f >> 5) * kGAStride + (f & 31)] = grow[kRadial + f];
    const float4 xi = g.pos[q];
    const int nr = min(nl.cnt_r[q], nl.cap_r);
    const int* lr = nl.nbr_r + (size_t)q * nl.cap_r;
    __syncwarp();

    float gix = 0.f, giy = 0.f, giz = 0.f;
    // ---- radial: lane per neighbour ----
    for (int t = lane; t < nr; t += 32) {
      const int j = lr[t];
      const float3 d = disp(xi, g.pos[j], c);
      const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
      const float fc = 0.5f * cospif(r / c.Rcr) + 0.5f;
      const float dfc = -0.5f * kPi / c.Rcr * sinpif(r / c.Rcr);
      const float* gs = gR + g.species[j] * kShfR;
      float dEdr = 0.f;
#pragma unroll
      for (int k = 0; k < kShfR; ++k) {
        const float x = r - c.ShfR[k];
        const float e = expf(-c.EtaR * x * x);
        dEdr = fmaf(gs[k] * 0.25f * e, fmaf(-2.f * c.EtaR * x, fc, dfc), dEdr);
      }
      const float s = dEdr / r;
      sg[3 * t + 0] = s * d.x;
      sg[3 * t + 1] = s * d.y;
      sg[3 * t + 2] = s * d.z;
      gix -= s * d.x;
      giy -= s * d.y;
      giz -= s * d.z;
    }

    // ---- angular ----
    const int na = min(nl.cnt_a[q], nl.cap_a);
    {
      const int* la = nl.nbr_a + (size_t)q * nl.cap_a;
      const int* sa = nl.slot_a + (size_t)q * nl.cap_a;
      for (int t = lane; t < na; t += 32) {
        const int j = la[t];
        const float3 d = disp(xi, g.pos[j], c);
        const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        nb[t] = make_float4(d.x, d.y, d.z, r);
        nfc[t] = 0.5f * cospif(r / c.Rca) + 0.5f;
        ndfc[t] = -0.5f * kPi / c.Rca * sinpif(r / c.Rca);
        nsp[t] = g.species[j];
        nslot[t] = sa[t];
      }
    }
    __syncwarp();
    const int T = na * (na - 1) / 2;
    for (int base = 0; base < T; base += 32) {
      const int P = base + lane;
      const bool valid = P < T;
      int j = -1, k = -1;
      float gjx = 0.f, gjy = 0.f, gjz = 0.f, gkx = 0.f, gky = 0.f, gkz = 0.f;
      if (valid) {
        decode_pair(P, na, j, k);
        const float4 rj = nb[j], rk = nb[k];
        const float inv_jk = 1.f / (rj.w * rk.w);
        const float cost = (rj.x * rk.x + rj.y * rk.y + rj.z * rk.z) * inv_jk;
        const float cp = 0.95f * cost;
        const float sp = sqrtf(fmaxf(1.f - cp * cp, 1e-12f));
        const float fcj = nfc[j], fck = nfc[k];
        const float u = 0.5f * (rj.w + rk.w);
        const float* gp = gA + c.pair_index[nsp[j]][nsp[k]] * kGAStride;
        float A[kShfZ], dA[kShfZ];
#pragma unroll
        for (int z = 0; z < kShfZ; ++z) {
          const float b = fmaxf(0.5f * (1.f + cp * c.cosZ[z] + sp * c.sinZ[z]), 0.f);
          const float L = log2f(b);
          A[z] = 2.f * exp2f(c.Zeta * L);
          // dA/dcp = 2 Zeta b^(Zeta-1) db/dcp,  db/dcp = (cosZ - cp/sp sinZ) / 2
          dA[z] = c.Zeta * exp2f((c.Zeta - 1.f) * L) * (c.cosZ[z] - cp / sp * c.sinZ[z]);
        }
        float V = 0.f, dVdc = 0.f, dVdu = 0.f;
#pragma unroll
        for (int a = 0; a < kShfA; ++a) {
          const float x = u - c.ShfA[a];
          const float R = expf(-c.EtaA * x * x);
          float SA = 0.f, SdA = 0.f;
#pragma unroll
          for (int z = 0; z < kShfZ; ++z) {
            const float gv = gp[a * kShfZ + z];
            SA = fmaf(gv, A[z], SA);
            SdA = fmaf(gv, dA[z], SdA);
          }
          V = fmaf(R, SA, V);
          dVdc = fmaf(R, SdA, dVdc);
          dVdu = fmaf(-2.f * c.EtaA * x * R, SA, dVdu);
        }
        const float fcjk = fcj * fck;
        const float dEdcos = 0.95f * fcjk * dVdc;
        const float dEdu = fcjk * dVdu;
        const float dEdrj = 0.5f * dEdu + V * ndfc[j] * fck;
        const float dEdrk = 0.5f * dEdu + V * fcj * ndfc[k];
        const float cj = cost / (rj.w * rj.w), ck = cost / (rk.w * rk.w);
        const float ej = dEdrj / rj.w, ek = dEdrk / rk.w;
        gjx = dEdcos * (rk.x * inv_jk - cj * rj.x) + ej * rj.x;
        gjy = dEdcos * (rk.y * inv_jk - cj * rj.y) + ej * rj.y;
        gjz = dEdcos * (rk.z * inv_jk - cj * rj.z) + ej * rj.z;
        gkx = dEdcos * (rj.x * inv_jk - ck * rk.x) + ek * rk.x;
        gky = dEdcos * (rj.y * inv_jk - ck * rk.y) + ek * rk.y;
        gkz = dEdcos * (rj.z * inv_jk - ck * rk.z) + ek * rk.z;
        gix -= gjx + gkx;
        giy -= gjy + gky;
        giz -= gjz + gkz;
        const int sk = nslot[k];
        if (sk < nl.cap_r) {
          atomicAdd(&sg[3 * sk + 0], gkx);
          atomicAdd(&sg[3 * sk + 1], gky);
          atomicAdd(&sg[3 * sk + 2], gkz);
        }
      }
      // j side: lanes sharing j are contiguous -> segmented inclusive scan.
      const int key = valid ? j : -1 - lane;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float ox = __shfl_up_sync(0xffffffffu, gjx, off);
        const float oy = __shfl_up_sync(0xffffffffu, gjy, off);
        const float oz = __shfl_up_sync(0xffffffffu, gjz, off);
        const int ok = __shfl_up_sync(0xffffffffu, key, off);
        if (lane >= off && ok == key) {
          gjx += ox;
          gjy += oy;
          gjz += oz;
        }
      }
      const int next = __shfl_down_sync(0xffffffffu, key, 1);
      if (valid && (lane == 31 || next != key)) {
        const int sj = nslot[j];
        if (sj < nl.cap_r) {
          atomicAdd(&sg[3 * sj + 0], gjx);
          atomicAdd(&sg[3 * sj + 1], gjy);
          atomicAdd(&sg[3 * sj + 2], gjz);
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      gix += __shfl_xor_sync(0xffffffffu, gix, o);
      giy += __shfl_xor_sync(0xffffffffu, giy, o);
      giz += __shfl_xor_sync(0xffffffffu, giz, o);
    }
    __syncwarp();
    for (int t = lane; t < nr; t += 32)
      add_force(acc_w, lr[t] - a0, orig, lr[t], F, sg[3 * t], sg[3 * t + 1], sg[3 * t + 2]);
    if (lane == 0) add_force(acc_w, q - a0, orig, q, F, gix, giy, giz);
    __syncwarp();
  }
  if (smem_acc) {
    __syncthreads();
    for (int t = threadIdx.x; t < n_mol * 3; t += blockDim.x) {
      double s = 0.0;
      for (int ww = 0; ww < nwarps; ++ww) s += accm[(size_t)ww * smem_atoms_max * 3 + t];
      if (s != 0.0) atomicAdd(F + 3 * (size_t)orig[a0 + t / 3] + (t % 3), -s);
    }
  }
}

}  // namespace

void launch_neighbors(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                      unsigned* status, cudaStream_t s) {
  if (g.n_atoms <= 0) return;
  const int threads = 256;
  const int blocks = (int)(((long)g.n_atoms * 32 + threads - 1) / threads);
  k_neighbors<<<blocks, threads, 0, s>>>(g, nl, c, status);
}

size_t aev_fwd_smem_bytes(int cap_a, int warps) {
  return (size_t)warps * aev_fwd_warp_floats(cap_a) * sizeof(float);
}

size_t aev_adj_smem_bytes(int cap_r, int cap_a, int warps, int mol_atoms_smem_max) {
  return (size_t)warps * mol_atoms_smem_max * 3 * sizeof(double) +
         (size_t)warps * adj_warp_floats(cap_r, cap_a) * sizeof(float);
}

void launch_aev(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                const int* row_of_int, void* out, Prec prec, int warps, cudaStream_t s) {
  if (g.n_atoms <= 0) return;
  const int blocks = (g.n_atoms + warps - 1) / warps;
  const size_t smem = aev_fwd_smem_bytes(nl.cap_a, warps);
  switch (prec) {
    case Prec::F32:
      k_aev<float><<<blocks, warps * 32, smem, s>>>(g, nl, c, row_of_int, (float*)out);
      break;
    case Prec::BF16:
      k_aev<__nv_bfloat16><<<blocks, warps * 32, smem, s>>>(g, nl, c, row_of_int,
                                                           (__nv_bfloat16*)out);
      break;
    case Prec::F16:
      k_aev<__half><<<blocks, warps * 32, smem, s>>>(g, nl, c, row_of_int, (__half*)out);
      break;
  }
}

void launch_aev_adjoint(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                        const int* row_of_int, const float* dG, const int4* work, int n_work,
                        const int* orig, double* F, int warps, int mol_atoms_smem_max,
                        cudaStream_t s) {
  if (n_work <= 0) return;
  const size_t smem = aev_adj_smem_bytes(nl.cap_r, nl.cap_a, warps, mol_atoms_smem_max);
  k_aev_adjoint<<<n_work, warps * 32, smem, s>>>(g, nl, c, row_of_int, dG, work, orig, F,
                                                mol_atoms_smem_max);
}

// Raises (never lowers) the dynamic shared-memory limits of the featurizer
// kernels, so handles of different sizes can coexist in one process.
cudaError_t aev_set_smem_limits(size_t fwd_bytes, size_t adj_bytes) {
  static size_t fwd_max = 0, adj_max = 0;
  fwd_bytes = fwd_max = fwd_bytes > fwd_max ? fwd_bytes : fwd_max;
  adj_bytes = adj_max = adj_bytes > adj_max ? adj_bytes : adj_max;
  cudaError_t e;
  e = cudaFuncSetAttribute(k_aev<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_aev<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fwd_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_aev<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_aev_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)adj_bytes);
}

}  // namespace nnp
