// aev.cu -- neighbour lists, the ANI featurizer and its reverse pass.
//
// Neighbour search: one CTA per chunk of 64 centres of a molecule, the
// molecule's positions staged in shared memory; one warp per centre scans
// the molecule 32 candidates at a time; a ballot and a prefix popcount
// compact the accepted candidates in ascending internal index, so every list
// is sorted and therefore grouped by element.  The cutoff test is FP32 with
// an FP64 recheck of the exact squared distance inside a 1e-4 relative guard
// band, which makes the pair sets identical to an FP64 evaluation.  (The
// one-warp-per-centre kernel without staging serves the allocation-free
// entry point.)
//
// Featurizer (the modified Behler-Parrinello functions the paper names in
// Sec. 1; Sec. 2 "Optimization" describes the custom CUDA featurizer): one
// warp per centre.  Radial terms: lanes = 16 shifts x 2 neighbours, summed
// into a per-warp shared-memory row (each lane owns one column: no atomics).
// Angular terms: neighbour pairs enumerated block by block (species pair),
// each block padded to a multiple of 4 pairs and decoded in closed form
// (rectangle, or folded triangle for one element); two phases per 32 pairs:
// (1) lane per pair computes the 4 angle factors and 8 distance factors;
// (2) lane per feature (8 x 4) walks the 8 groups of 4 pairs and accumulates
// R_a * A_z into its block in registers, writing the block when the next
// one starts.
//
// Reverse pass: one warp per centre, lane per neighbour (radial) and lane per
// pair (angular, folded-triangle order); per-neighbour gradients gather in
// shared memory (the j side of a run of pairs by a segmented warp scan), then
// go to a per-warp FP64 accumulator of the molecule or to FP64 global
// atomics.  Centres with more angular neighbours than the main launch stages
// are deferred to a second launch.
#include <mutex>

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
        if (sl < nl.cap_a) la[sl] = j;
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

// The same search with one CTA per work item (a chunk of up to kNbrChunk
// centres of one molecule): the molecule's positions are staged in shared
// memory once (when they fit) and each warp takes centres of the chunk.
constexpr int kNbrChunk = 64;
constexpr int kNbrWarps = 8;
constexpr int kNbrStageMax = 2048;  // atoms of a molecule staged in shared memory

__global__ void __launch_bounds__(32 * kNbrWarps) k_neighbors_mol(Geometry g, NeighborLists nl,
                                                                  AevConst c, const int4* __restrict__ work,
                                                                  unsigned* status) {
  extern __shared__ float4 spos[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the featurizer may launch
  const int4 w = work[blockIdx.x];
  const int a0 = w.x, n = w.y, a1 = a0 + n;
  const bool staged = n <= kNbrStageMax;
  if (staged)
    for (int t = threadIdx.x; t < n; t += blockDim.x) spos[t] = g.pos[a0 + t];
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int q = w.z + warp; q < w.w; q += kNbrWarps) {
    const float4 xi = staged ? spos[q - a0] : g.pos[q];
    int nr = 0, na = 0;
    int* lr = nl.nbr_r + (size_t)q * nl.cap_r;
    int* la = nl.nbr_a + (size_t)q * nl.cap_a;
    for (int base = a0; base < a1; base += 32) {
      const int j = base + lane;
      bool inR = false, inA = false;
      if (j < a1 && j != q) {
        const float4 xj = staged ? spos[j - a0] : g.pos[j];
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
          if (sl < nl.cap_a) la[sl] = j;
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
}

// Pair P (0 <= P < n(n-1)/2) of n items, j < k, in the folded-triangle
// order: rows of width W = n - 1 (n even) or n (n odd); row a holds the pairs
// (a, a+1 .. n-1) followed by those of row n-1-a (n even) or n-2-a (n odd),
// so each row is two runs of constant j.  invW = 1/W as a float.
__device__ __forceinline__ void fold_pair(int P, int n, int W, float invW, int& j, int& k) {
  int q = (int)((float)P * invW);  // P / W, then exact
  int c = P - q * W;
  if (c < 0) {
    --q;
    c += W;
  } else if (c >= W) {
    ++q;
    c -= W;
  }
  const int span = n - 1 - q;
  j = c < span ? q : n - 1 - q - (n & 1);
  k = c < span ? q + 1 + c : j + 1 + (c - span);
}

template <typename T> __device__ __forceinline__ T cvt_out(float v);
template <> __device__ __forceinline__ float cvt_out<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half cvt_out<__half>(float v) { return __float2half_rn(v); }
__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }

// Per-warp shared memory of the forward kernel (floats):
//   buf[12][36] (the radial accumulators R2[2][112] alias it) | meta (ints): block
//   prefix bpre[32], block decode records bm int4[28] and be int2[28], group
//   start gs[8], group count gn[8] |
//   staging union: radial {rd, rfc, rsp}[cap_r]  or  angular {avec float4, afc, asp}[cap_a]
constexpr int kBufStride = 36;  // phase-1 factor rows: 16-byte aligned, bank-spread
constexpr int kMeta = 32 + 4 * kPairBlocks + 2 * kPairBlocks + 16;
__host__ __device__ constexpr int aev_fwd_warp_floats(int cap_r, int cap_a) {
  return 12 * kBufStride + kMeta + (3 * cap_r > 6 * cap_a ? 3 * cap_r : 6 * cap_a);
}


// The SFU base-2 exponential and logarithm, denormals flushed to zero (values
// below 2^-126 only ever multiply other factors here).
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_ftz(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// b^N for a compile-time N >= 0 by repeated squaring (ceil(log2 N) squarings
// and a multiplication per set bit).  Each rounding is unbiased, and the
// relative error stays near N times that of b.
template <int N> __device__ __forceinline__ float powi(float b) {
  if constexpr (N == 0) {
    return 1.f;
  } else if constexpr (N == 1) {
    return b;
  } else {
    const float h = powi<N / 2>(b);
    return (N & 1) ? h * h * b : h * h;
  }
}

// Packed FP32 arithmetic: two values per instruction, per component the
// roundings of the scalar operation (so the same results as the scalar code).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 ex2_ftz2(float2 x) { return make_float2(ex2_ftz(x.x), ex2_ftz(x.y)); }
__device__ __forceinline__ float2 lg2_ftz2(float2 x) { return make_float2(lg2_ftz(x.x), lg2_ftz(x.y)); }
template <int N> __device__ __forceinline__ float2 powi2(float2 b) {
  if constexpr (N == 0) {
    return f2(1.f);
  } else if constexpr (N == 1) {
    return b;
  } else {
    const float2 h = powi2<N / 2>(b);
    return (N & 1) ? mul2(mul2(h, h), b) : mul2(h, h);
  }
}
// 2^(-y^2) of two Gaussian arguments y = fma(r, c_hi, -s_hi) + fma(r, c_lo, -s_lo)
__device__ __forceinline__ float2 gauss2(float r, float c_hi, float c_lo, float s_hi0, float s_hi1,
                                         float s_lo0, float s_lo1, float2& y) {
  y = add2(fma2(f2(r), f2(c_hi), make_float2(-s_hi0, -s_hi1)), fma2(f2(r), f2(c_lo), make_float2(-s_lo0, -s_lo1)));
  return ex2_ftz2(mul2(make_float2(-y.x, -y.y), y));
}

// Species pair (s, t), s <= t, of each block, row-major upper triangle: the
// 28 blocks of seven elements, then the 10 of four.
__constant__ unsigned char kBlkS[kPairBlocks + 10] = {0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3,
                                                      3, 3, 3, 4, 4, 4, 5, 5, 6, 0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
__constant__ unsigned char kBlkT[kPairBlocks + 10] = {0, 1, 2, 3, 4, 5, 6, 1, 2, 3, 4, 5, 6, 2, 3, 4, 5, 6, 3,
                                                      4, 5, 6, 4, 5, 6, 5, 6, 6, 0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
template <int NS> __device__ __forceinline__ int blk_s(int b) {
  static_assert(NS == 7 || NS == 4, "tables of seven and of four elements");
  return kBlkS[(NS == 7 ? 0 : kPairBlocks) + b];
}
template <int NS> __device__ __forceinline__ int blk_t(int b) {
  return kBlkT[(NS == 7 ? 0 : kPairBlocks) + b];
}

// Index of the unordered species pair {s, t} in the row-major upper triangle
// of NS elements.
template <int NS> __device__ __forceinline__ int pair_block(int s, int t) {
  const int a = min(s, t), b = max(s, t);
  return a * NS - (a * (a - 1)) / 2 + (b - a);
}

// Element groups of an element-sorted angular neighbour list and the prefix
// of the block-major pair enumeration, each block padded to a multiple of 4
// pairs (the padding pairs contribute zero).  cnt_s: on lanes 0..NS-1 the size
// of element group s.  Writes gs[NS] (group starts), gn[NS] (sizes), bpre[NP+1]
// (first pair of each block, bpre[NP] = padded number of pairs) and for each
// block its decode record: bm[b] = (row width W, first list position of the
// j group, of the k group, pairs), be[b] = (n for a same-element block, else
// 0; bits of 1/W).  A block of two elements is a rectangle: pair l is (row
// l / W, column l % W).  A same-element block of n atoms is its upper
// triangle folded into a rectangle of width W = n - 1 (n even) or n (n odd):
// row a holds the n-1-a pairs (a, a+1..) followed by the pairs of row
// n-1-a (n even) or n-2-a (n odd), so that every row has W pairs.  Call with
// the whole warp, then __syncwarp before reading.
template <int NS>
__device__ __forceinline__ void angular_blocks(int cnt_s, int lane, int* gs, int* gn, int* bpre,
                                               int4* bm, int2* be) {
  constexpr int NP = NS * (NS + 1) / 2;
  const unsigned FULL = 0xffffffffu;
  int start = cnt_s;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int v = __shfl_up_sync(FULL, start, o);
    if (lane >= o) start += v;
  }
  start -= cnt_s;
  if (lane < NS) {
    gs[lane] = start;
    gn[lane] = cnt_s;
  }
  const int bs = lane < NP ? blk_s<NS>(lane) : 0, bt = lane < NP ? blk_t<NS>(lane) : 0;
  const int ns = __shfl_sync(FULL, cnt_s, bs), nt = __shfl_sync(FULL, cnt_s, bt);
  const int gss = __shfl_sync(FULL, start, bs), gst = __shfl_sync(FULL, start, bt);
  const int size = lane < NP ? (bs == bt ? ns * (ns - 1) / 2 : ns * nt) : 0;
  if (lane < NP) {
    const int w = bs == bt ? ((ns & 1) ? ns : ns - 1) : nt;
    const int wd = w > 0 ? w : 1;
    bm[lane] = make_int4(wd, gss, gst, size);
    be[lane] = make_int2(bs == bt ? ns : 0, __float_as_int(1.f / (float)wd));
  }
  int incl = (size + 3) & ~3;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane < NP) bpre[lane + 1] = incl;
  if (lane == 0) bpre[0] = 0;
}

// Pair P of the (padded) block-major enumeration: its block and the list
// positions j < k of its two neighbours, or j = -1 for a padding pair.
// b0: the block holding the warp's first pair of this iteration, base: that
// pair (the iteration covers base .. base + 31).
template <int NP>
__device__ __forceinline__ int decode_block_pair(int P, int b0, int base, const int* bpre, const int4* bm,
                                                 const int2* be, int& j, int& k) {
  // the last block starting at or before P among those starting in the
  // iteration's window (a uniform walk over the window's few block starts)
  int b = b0;
  for (int bb = b0 + 1; bb < NP && bpre[bb] < base + 32; ++bb) b = bpre[bb] <= P ? bb : b;
  const int l = P - bpre[b];
  const int4 m = bm[b];  // W, j-group start, k-group start, pairs
  const int2 e = be[b];  // n (same-element block) or 0, 1/W
  if (l >= m.w) {
    j = k = -1;
    return b;
  }
  int q = (int)((float)l * __int_as_float(e.y));  // l / W, then exact
  int c = l - q * m.x;
  if (c < 0) {
    --q;
    c += m.x;
  } else if (c >= m.x) {
    ++q;
    c -= m.x;
  }
  const int n = e.x;
  if (n == 0) {  // two elements: rectangle
    j = m.y + q;
    k = m.z + c;
  } else {  // one element: folded triangle (as fold_pair), row q
    const int span = n - 1 - q;
    const int jj = c < span ? q : n - 1 - q - (n & 1);
    const int kk = c < span ? q + 1 + c : jj + 1 + (c - span);
    j = m.y + jj;
    k = m.y + kk;
  }
  return b;
}

// The angular features of a centre are sums over unordered neighbour pairs.
// Pairs are enumerated block-major: species-pair block b = (s, t) holds every
// pair with one neighbour of element s and one of element t (the neighbour
// list is sorted by element, so each element is one contiguous group), and
// the blocks follow each other in feature order.  Each block is then one
// contiguous run of pairs, accumulated once and written once; padded to a
// multiple of 4 pairs, every run starts 16-byte aligned in the factor rows.
// With kSplit each feature v is written as hi = round(v) in the row's first
// kPad columns and lo = round(v - hi) in the next kPad (16-bit outputs).
// Shape: the model's elements and angular grid (NA distance x NZ angle
// shifts, NA x NZ = 32 features per block).
template <typename TOut, bool kSplit, typename Shape>
__global__ void k_aev(Geometry g, NeighborLists nl, AevConst c, const int* __restrict__ row_of_int,
                      TOut* __restrict__ out) {
  constexpr int NS = Shape::NS, NA = Shape::NA, NZ = Shape::NZ, NP = Shape::kNP;
  constexpr int kRad = Shape::kRad, kFeat = Shape::kFeat, kPad = Shape::kPad;
  extern __shared__ __align__(16) float smem[];
  const unsigned FULL = 0xffffffffu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + warp;
  // the first-layer product may launch (and run its prologue) once every CTA
  // of this grid has started; it waits for this grid's results
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");  // neighbour lists of the kernel before
  if (q >= g.n_atoms) return;  // warp-uniform; no block-level barriers below
  float* buf = smem + (size_t)warp * aev_fwd_warp_floats(nl.cap_r, nl.cap_a);  // [12][36]
  float* R2 = buf;                                       // [2][kRad], radial phase only
  int* bpre = reinterpret_cast<int*>(buf + 12 * kBufStride);  // [29] block prefix
  int4* bm = reinterpret_cast<int4*>(bpre + 32);         // [28] block decode records
  int2* be = reinterpret_cast<int2*>(bm + kPairBlocks);  // [28]
  int* gs = reinterpret_cast<int*>(be + kPairBlocks);    // [7] group start
  int* gn = gs + 8;                                      // [7] group size
  float* U = buf + 12 * kBufStride + kMeta;              // staging union (16-byte aligned)
  float* rd = U;
  float* rfc = rd + nl.cap_r;
  int* rsp = reinterpret_cast<int*>(rfc + nl.cap_r);
  float4* avec = reinterpret_cast<float4*>(U);
  float* afc = reinterpret_cast<float*>(avec + nl.cap_a);
  int* asp = reinterpret_cast<int*>(afc + nl.cap_a);
  TOut* dst = out + (size_t)row_of_int[q] * (kSplit ? 2 : 1) * kPad;
  auto put = [&](int f, float v) {
    const TOut hi = cvt_out<TOut>(v);
    dst[f] = hi;
    if (kSplit) dst[kPad + f] = cvt_out<TOut>(v - to_float(hi));
  };

  for (int f = lane; f < 2 * kRad; f += 32) R2[f] = 0.f;
  const float4 xi = g.pos[q];

  // ---- radial: stage the neighbours (lane-parallel loads), then lane =
  //      (neighbour parity, shift), each lane owning one accumulator column ----
  const int nr = min(nl.cnt_r[q], nl.cap_r);
  {
    const int* lr = nl.nbr_r + (size_t)q * nl.cap_r;
    for (int t = lane; t < nr; t += 32) {
      const int j = lr[t];
      const float4 xj = g.pos[j];  // w: the element index
      const float3 d = disp(xi, xj, c);
      const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
      rd[t] = r;
      rfc[t] = 0.125f * cospif(r / c.Rcr) + 0.125f;  // fc / 4 (the radial prefactor)
      rsp[t] = __float_as_int(xj.w);
    }
  }
  __syncwarp();
  {
    const int half = lane >> 4, k = lane & 15;
    const float shs = c.ShfRs[k], shsl = c.ShfRsl[k];
    float* acc = R2 + half * kRad;
    for (int t = half; t < nr; t += 2) {
      // exp(-EtaR (r - ShfR)^2) = 2^(-y^2), constants as hi + lo pairs
      const float y = fmaf(rd[t], c.sqEtaR, -shs) + fmaf(rd[t], c.sqEtaRl, -shsl);
      acc[rsp[t] * kShfR + k] += ex2_ftz(-y * y) * rfc[t];
    }
  }
  __syncwarp();
  for (int f = lane; f < kRad; f += 32) put(f, R2[f] + R2[kRad + f]);
  __syncwarp();  // R2 and the radial staging are dead from here on

  // ---- angular staging and the element groups of the list ----
  const int na = min(nl.cnt_a[q], nl.cap_a);
  int cnt_s = 0;  // lane s < NS: size of element group s
  {
    const int* la = nl.nbr_a + (size_t)q * nl.cap_a;
    for (int base = 0; base < na; base += 32) {
      const int t = base + lane;
      int sp = -1;
      if (t < na) {
        const int j = la[t];
        const float4 xj = g.pos[j];
        const float3 d = disp(xi, xj, c);
        const float r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        avec[t] = make_float4(d.x, d.y, d.z, r);
        afc[t] = 0.5f * cospif(r / c.Rca) + 0.5f;
        sp = __float_as_int(xj.w);
        asp[t] = sp;
      }
#pragma unroll
      for (int e = 0; e < NS; ++e) {
        const int n_e = __popc(__ballot_sync(FULL, sp == e));
        if (lane == e) cnt_s += n_e;
      }
    }
  }
  angular_blocks<NS>(cnt_s, lane, gs, gn, bpre, bm, be);
  __syncwarp();
  const int T = bpre[NP];

  // ---- angular, 32 neighbour pairs at a time ----
  const int fa = lane / NZ, fz = lane % NZ;
  float acc = 0.f;
  int pcur = -1;  // block being accumulated; blocks before it are written
  int b0 = 0;  // block holding the iteration's first pair
  for (int base = 0; base < T; base += 32) {
    while (bpre[b0 + 1] <= base) ++b0;  // uniform; bpre[NP] = T > base
    const int P = base + lane;
    const bool valid = P < T;
    int pl = -1;
    if (valid) {
      // phase 1: this lane's pair -> NA distance factors, NZ angle factors
      int j, k;
      const int b = decode_block_pair<NP>(P, b0, base, bpre, bm, be, j, k);
      if (j >= 0) {
        const float4 rj = avec[j], rk = avec[k];
        const float cost = __fdividef(rj.x * rk.x + rj.y * rk.y + rj.z * rk.z, rj.w * rk.w);
        const float cp = 0.95f * cost;
        const float sp = sqrtf(fmaxf(1.f - cp * cp, 0.f));
        const float fcjk = 2.f * afc[j] * afc[k];
        const float u = 0.5f * (rj.w + rk.w);
#pragma unroll
        for (int a = 0; a < NA; a += 2) {
          // 2^(-y^2) = exp(-EtaA (u - ShfA)^2), two shifts at a time
          float2 y;
          const float2 R = gauss2(u, c.sqEtaA, c.sqEtaAl, c.ShfAs[a], c.ShfAs[a + 1], c.ShfAsl[a], c.ShfAsl[a + 1], y);
          buf[a * kBufStride + lane] = R.x;
          buf[(a + 1) * kBufStride + lane] = R.y;
        }
#pragma unroll
        for (int z = 0; z < NZ; z += 2) {
          // t = 1 + cos(theta' - ThetaS): ((1 + cos) / 2)^Zeta = 2^(Zeta (lg2 t - 1)),
          // or (t / 2)^Zeta by multiplication for an integer Zeta
          const float2 t0 = fma2(f2(sp), make_float2(c.sinZ[z], c.sinZ[z + 1]),
                                 fma2(f2(cp), make_float2(c.cosZ[z], c.cosZ[z + 1]), f2(1.f)));
          const float2 t = make_float2(fmaxf(t0.x, 0.f), fmaxf(t0.y, 0.f));
          float2 A;
          if constexpr (Shape::kZetaInt > 0) A = powi2<Shape::kZetaInt>(mul2(f2(0.5f), t));
          else A = ex2_ftz2(fma2(f2(c.Zeta), lg2_ftz2(t), f2(-c.Zeta)));
          const float2 Af = mul2(A, f2(fcjk));
          buf[(NA + z) * kBufStride + lane] = Af.x;
          buf[(NA + z + 1) * kBufStride + lane] = Af.y;
        }
      } else {  // padding pair: zero factors
#pragma unroll
        for (int f = 0; f < NA + NZ; ++f) buf[f * kBufStride + lane] = 0.f;
      }
      pl = b;
    } else {  // past the last pair: zero factors, so phase 2 can walk all 8 groups
#pragma unroll
      for (int f = 0; f < NA + NZ; ++f) buf[f * kBufStride + lane] = 0.f;
    }
    // phase 2: lane = feature (a, z).  Blocks are padded to multiples of 4
    // pairs, so each group of 4 pairs lies in one block: walk the 8 groups
    // (groups past the last pair hold zeros and add nothing), writing the
    // accumulated block where the next one starts.
    const int prev = __shfl_up_sync(FULL, pl, 1);
    const unsigned starts = __ballot_sync(FULL, valid && (lane == 0 || prev != pl));
    __syncwarp();
    const float4* ra4 = reinterpret_cast<const float4*>(buf + fa * kBufStride);
    const float4* za4 = reinterpret_cast<const float4*>(buf + (NA + fz) * kBufStride);
#pragma unroll
    for (int gi = 0; gi < 8; ++gi) {
      if ((starts >> (4 * gi)) & 1u) {
        const int p = __shfl_sync(FULL, pl, 4 * gi);
        if (p != pcur) {  // block pcur is complete: write it, and zeros for empty blocks
          if (pcur >= 0) put(kRad + pcur * 32 + lane, acc);
          for (int e = pcur + 1; e < p; ++e) put(kRad + e * 32 + lane, 0.f);
          acc = 0.f;
          pcur = p;
        }
      }
      const float4 r4 = ra4[gi], z4 = za4[gi];
      acc = fmaf(r4.x, z4.x, acc);
      acc = fmaf(r4.y, z4.y, acc);
      acc = fmaf(r4.z, z4.z, acc);
      acc = fmaf(r4.w, z4.w, acc);
    }
    __syncwarp();
  }
  if (pcur >= 0) put(kRad + pcur * 32 + lane, acc);
  for (int e = pcur + 1; e < NP; ++e) put(kRad + e * 32 + lane, 0.f);
  if (lane < kPad - kFeat) put(kFeat + lane, 0.f);
}

// ---------------------------------------------------------------------------
// Reverse pass.

constexpr int kGAStride = 36;  // padded row of an angular block (16-byte aligned, bank spread)

// Per-warp shared memory of the reverse pass (floats):
//   gR[7][20] | gA[28][36] | nb float4[cap_a][2] | sg[cap_a][3]
// nb[t] = {(unit vector, distance), (fc, dfc/dr, 1 / distance, species bits)}
// (rows padded to 20 and 36 floats: 16-byte aligned, and the rows that a
// warp's 16-byte loads hit at once fall in distinct banks)
constexpr int kGRStride = 20;
__host__ __device__ constexpr int adj_warp_floats(int /*cap_r*/, int cap_a) {
  return kSpecies * kGRStride + kPairBlocks * kGAStride + 11 * cap_a;
}

// Adds a gradient to the force of atom a_glob (internal index): into the
// warp's own FP64 accumulator of the molecule, or with FP64 atomics straight
// into the forces when the molecule is too large for shared memory.
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

// Per-warp staging capacity (angular neighbours) of the reverse pass's main
// launch; centres with more angular neighbours are deferred to a second
// launch with staging for the full capacity, so the common case keeps its
// shared memory, and with it the occupancy, small.
constexpr int kAdjStage = 64;

// Reverse pass of the featurizer: given dE/dG of every atom, the forces.
// Main pass (pass 0): one work item (CTA) = a chunk of centres of one
// molecule; warps take centres as they free up; a centre with more than
// stage_cap angular neighbours is appended to the overflow list ovf
// (ovf[0] = count, ovf[1..] = centres).  Overflow pass (pass 1): the CTAs
// share out the listed centres, staging for stage_cap = the full capacity,
// forces by FP64 atomics.  Per centre: radial terms lane per neighbour,
// angular terms lane per pair; each pair's gradients go to per-neighbour
// accumulators in shared memory
// (the lanes of a chunk that share the first neighbour are reduced by a
// segmented scan first), then to the warp's FP64 accumulator of the molecule.
template <typename Shape>
__global__ void __launch_bounds__(128, 7) k_aev_adjoint(Geometry g, NeighborLists nl, AevConst c,
                              const int* __restrict__ row_of_int, const float* __restrict__ dG,
                              const int4* __restrict__ work, const int* __restrict__ orig,
                              double* __restrict__ F, int smem_atoms_max, int stage_cap,
                              int* __restrict__ ovf, int pass) {
  constexpr int NS = Shape::NS, NA = Shape::NA, NZ = Shape::NZ;
  constexpr int kRad = Shape::kRad, kFeat = Shape::kFeat, kPad = Shape::kPad;
  static_assert(kFeat / 4 <= 8 * 32, "dE/dG row: at most 8 float4 per lane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned FULL = 0xffffffffu;
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 w = pass == 0 ? work[blockIdx.x] : make_int4(0, 0, 0, 0);
  const int a0 = w.x, n_mol = w.y, q0 = w.z, q1 = w.w;
  const bool smem_acc = pass == 0 && n_mol <= smem_atoms_max;
  double* accm = reinterpret_cast<double*>(smem_raw);  // [nwarps][smem_atoms_max][3]
  float* gR = reinterpret_cast<float*>(accm + (size_t)nwarps * smem_atoms_max * 3) +
              (size_t)warp * adj_warp_floats(nl.cap_r, stage_cap);
  float* gA = gR + kSpecies * kGRStride;  // [NP <= 28][36]
  float4* nb = reinterpret_cast<float4*>(gA + kPairBlocks * kGAStride);  // [stage_cap][2]
  float* sg = reinterpret_cast<float*>(nb + 2 * stage_cap);                // [stage_cap][3]
  double* acc_w = smem_acc ? accm + (size_t)warp * smem_atoms_max * 3 : nullptr;

  __shared__ int next_centre;  // centres (or overflow-list entries) handed to warps as they free up
  if (threadIdx.x == 0) next_centre = pass == 0 ? q0 : 0;
  if (smem_acc)
    for (int t = threadIdx.x; t < nwarps * smem_atoms_max * 3; t += blockDim.x) accm[t] = 0.0;
  __syncthreads();
  // dE/dG (and the overflow list) come from the kernels before this one
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int n_ovf = pass == 0 ? 0 : ovf[0];

  const float inv_rcr = 1.f / c.Rcr, inv_rca = 1.f / c.Rca;
  const float dfc_r = -0.5f * kPi * inv_rcr, dfc_a = -0.5f * kPi * inv_rca;  // d fc / dr = dfc_x sin(pi r / Rc)
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(&next_centre, 1);
    q = __shfl_sync(FULL, q, 0);
    if (pass == 0) {
      if (q >= q1) break;
    } else {
      const int e = blockIdx.x + gridDim.x * q;  // overflow-list entry
      if (e >= n_ovf) break;
      q = ovf[1 + e];
    }
    const int na = min(nl.cnt_a[q], nl.cap_a);
    if (na > stage_cap) {  // main pass only: defer to the overflow pass
      if (lane == 0) ovf[1 + atomicAdd(ovf, 1)] = q;
      continue;
    }
    {
      // dE/dG row: kFeat / 4 float4 (252 of ANI-2x, 96 of ANI-1x), up to 8
      // per lane, loads issued together
      const float4* grow = reinterpret_cast<const float4*>(dG + (size_t)row_of_int[q] * kPad);
      float4 v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int f4 = lane + 32 * i;
        if (f4 < kFeat / 4) v[i] = __ldg(grow + f4);
      }
      // 16-byte stores: radial float4 f4 < kRad / 4 is (species f4 / 4, shifts
      // 4 (f4 % 4) ..), angular float4 f4 is (block (f4 - kRad / 4) / 8,
      // features 4 ((f4 - kRad / 4) % 8) ..)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int f4 = lane + 32 * i;
        if (f4 >= kFeat / 4) continue;
        float* d = f4 < kRad / 4 ? gR + (f4 >> 2) * kGRStride + 4 * (f4 & 3)
                                 : gA + ((f4 - kRad / 4) >> 3) * kGAStride + 4 * ((f4 - kRad / 4) & 7);
        *reinterpret_cast<float4*>(d) = v[i];
      }
    }
    const float4 xi = g.pos[q];
    float gix = 0.f, giy = 0.f, giz = 0.f;

    // ---- angular staging (first: its loads overlap the dE/dG row's) ----
    const int* la = nl.nbr_a + (size_t)q * nl.cap_a;
    for (int t = lane; t < na; t += 32) {
      const int j = la[t];
      const float4 xj = g.pos[j];
      const float3 d = disp(xi, xj, c);
      const float ir = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
      const float r = (d.x * d.x + d.y * d.y + d.z * d.z) * ir;
      nb[2 * t] = make_float4(d.x * ir, d.y * ir, d.z * ir, r);
      float sn, cs;
      sincospif(r * inv_rca, &sn, &cs);
      nb[2 * t + 1] = make_float4(0.5f * cs + 0.5f, dfc_a * sn, ir, xj.w);  // w: element index bits
      sg[3 * t] = sg[3 * t + 1] = sg[3 * t + 2] = 0.f;
    }
    __syncwarp();

    // ---- radial: lane per neighbour, straight into the molecule accumulator ----
    {
      const int nr = min(nl.cnt_r[q], nl.cap_r);
      const int* lr = nl.nbr_r + (size_t)q * nl.cap_r;
      for (int t = lane; t < nr; t += 32) {
        const int j = lr[t];
        const float4 xj = g.pos[j];
        const float3 d = disp(xi, xj, c);
        const float ir = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        const float r = (d.x * d.x + d.y * d.y + d.z * d.z) * ir;
        float sn, cs;
        sincospif(r * inv_rcr, &sn, &cs);
        const float fc = 0.5f * cs + 0.5f;
        const float dfc = dfc_r * sn;
        // d(e fc)/dr / e = -2 EtaR (r - ShfR) fc + dfc = afc y + dfc, y = sqEtaR (r - ShfR)
        const float afc = c.gradR * fc;
        const float4* gsp = reinterpret_cast<const float4*>(gR + __float_as_int(xj.w) * kGRStride);
        float dEdr = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < kShfR / 4; ++k4) {
          const float4 g4 = gsp[k4];
          const float gk[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float y = fmaf(r, c.sqEtaR, -c.ShfRs[4 * k4 + h]) + fmaf(r, c.sqEtaRl, -c.ShfRsl[4 * k4 + h]);
            const float e = ex2_ftz(-y * y);  // exp(-EtaR (r - ShfR)^2)
            dEdr = fmaf(gk[h] * e, fmaf(afc, y, dfc), dEdr);
          }
        }
        const float s = 0.25f * dEdr * ir;
        gix -= s * d.x;
        giy -= s * d.y;
        giz -= s * d.z;
        add_force(acc_w, j - a0, orig, j, F, s * d.x, s * d.y, s * d.z);
      }
    }

    // ---- angular: lane per pair, pairs in folded-triangle order over the list
    //      (runs of equal j on contiguous lanes, k differing between lanes) ----
    const int T = na * (na - 1) / 2;
    const int fw = (na & 1) ? na : max(na - 1, 1);
    const float inv_fw = 1.f / (float)fw;
    for (int base = 0; base < T; base += 32) {
      const int P = base + lane;
      const bool valid = P < T;
      int j = -1, k = -1;
      float gjx = 0.f, gjy = 0.f, gjz = 0.f;
      if (valid) {
        fold_pair(P, na, fw, inv_fw, j, k);
        const float4 uj = nb[2 * j], uk = nb[2 * k];  // unit vectors, distances
        const float4 pj = nb[2 * j + 1], pk = nb[2 * k + 1];  // fc, dfc/dr, 1 / r, species
        const int b = pair_block<NS>(__float_as_int(pj.w), __float_as_int(pk.w));
        const float cost = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
        const float cp = 0.95f * cost;
        const float sp = sqrtf(fmaxf(1.f - cp * cp, 1e-12f));
        const float qs = __fdividef(cp, sp);
        const float fcj = pj.x, fck = pk.x;
        const float rjk = uj.w + uk.w;  // twice the angular distance u
        const float4* gp = reinterpret_cast<const float4*>(gA + b * kGAStride);
        // V = sum_a R_a sum_z g[a][z] A_z with R_a = exp(-EtaA (u - ShfA[a])^2)
        // = 2^(-y_a^2), y_a = sqEtaA (u - ShfA[a]), u = rjk / 2: the distance sums first,
        // GR[z] = sum_a R_a g[a][z] and GY[z] = sum_a y_a R_a g[a][z]
        float GR[NZ], GY[NZ];
#pragma unroll
        for (int z = 0; z < NZ; ++z) GR[z] = GY[z] = 0.f;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
          const float y = fmaf(rjk, c.hsqEtaA, -c.ShfAs[a]) + fmaf(rjk, c.hsqEtaAl, -c.ShfAsl[a]);
          const float R = ex2_ftz(-y * y);
          const float yR = y * R;
#pragma unroll
          for (int z4 = 0; z4 < NZ / 4; ++z4) {
            const float4 g4 = gp[a * (NZ / 4) + z4];  // g[a][4 z4 .. 4 z4 + 3]
            GR[4 * z4 + 0] = fmaf(R, g4.x, GR[4 * z4 + 0]);
            GR[4 * z4 + 1] = fmaf(R, g4.y, GR[4 * z4 + 1]);
            GR[4 * z4 + 2] = fmaf(R, g4.z, GR[4 * z4 + 2]);
            GR[4 * z4 + 3] = fmaf(R, g4.w, GR[4 * z4 + 3]);
            GY[4 * z4 + 0] = fmaf(yR, g4.x, GY[4 * z4 + 0]);
            GY[4 * z4 + 1] = fmaf(yR, g4.y, GY[4 * z4 + 1]);
            GY[4 * z4 + 2] = fmaf(yR, g4.z, GY[4 * z4 + 2]);
            GY[4 * z4 + 3] = fmaf(yR, g4.w, GY[4 * z4 + 3]);
          }
        }
        // angle factors, t = 2b = 1 + cp cosZ + sp sinZ: A = 2 b^Zeta = t pz
        // with pz = b^(Zeta-1) = 2^((Zeta-1)(lg2 t - 1)); dA/dcp = Zeta pz
        // (cosZ - cp/sp sinZ), Zeta applied once below
        float V = 0.f, dVdc = 0.f, dVdu = 0.f;
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
          const float t = fmaxf(fmaf(sp, c.sinZ[z], fmaf(cp, c.cosZ[z], 1.f)), 0.f);
          float pz;
          if constexpr (Shape::kZetaInt > 0) pz = powi<Shape::kZetaInt - 1>(0.5f * t);
          else pz = ex2_ftz(fmaf(c.Zeta - 1.f, lg2_ftz(t), 1.f - c.Zeta));
          const float A = t * pz;
          V = fmaf(GR[z], A, V);
          dVdu = fmaf(GY[z], A, dVdu);  // dV/du = gradA x this
          dVdc = fmaf(GR[z] * pz, fmaf(-qs, c.sinZ[z], c.cosZ[z]), dVdc);  // x Zeta
        }
        const float fcjk = fcj * fck;
        const float dEdcos = c.dcosA * fcjk * dVdc;
        const float hdEdu = c.hgradA * fcjk * dVdu;  // dE/du / 2 = dE/dr_j via u
        const float dEdrj = fmaf(V * fck, pj.y, hdEdu);
        const float dEdrk = fmaf(V * fcj, pk.y, hdEdu);
        // d cos / d r_j = (u_k - cos u_j) / |r_j|,  d |r_j| / d r_j = u_j, so
        // g_j = aj u_k + (dE/dr_j - aj cos) u_j with aj = dE/dcos / |r_j|
        const float aj = dEdcos * pj.z, ak = dEdcos * pk.z;
        const float bj = fmaf(-aj, cost, dEdrj), bk = fmaf(-ak, cost, dEdrk);
        gjx = fmaf(aj, uk.x, bj * uj.x);
        gjy = fmaf(aj, uk.y, bj * uj.y);
        gjz = fmaf(aj, uk.z, bj * uj.z);
        const float gkx = fmaf(ak, uj.x, bk * uk.x);
        const float gky = fmaf(ak, uj.y, bk * uk.y);
        const float gkz = fmaf(ak, uj.z, bk * uk.z);
        gix -= gjx + gkx;
        giy -= gjy + gky;
        giz -= gjz + gkz;
        atomicAdd(&sg[3 * k + 0], gkx);
        atomicAdd(&sg[3 * k + 1], gky);
        atomicAdd(&sg[3 * k + 2], gkz);
      }
      // j side: a run of consecutive lanes with the same j (the same j can
      // recur in a later block of the chunk: that is a separate run) is
      // reduced by a segmented inclusive scan; the run's last lane adds it.
      const int key = valid ? j : -1 - lane;
      const int prev_key = __shfl_up_sync(FULL, key, 1);
      const unsigned heads = __ballot_sync(FULL, lane == 0 || prev_key != key);
      const int head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // run start
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float ox = __shfl_up_sync(FULL, gjx, off);
        const float oy = __shfl_up_sync(FULL, gjy, off);
        const float oz = __shfl_up_sync(FULL, gjz, off);
        if (lane - off >= head) {
          gjx += ox;
          gjy += oy;
          gjz += oz;
        }
      }
      const bool run_end = lane == 31 || ((heads >> (lane + 1)) & 1u);
      if (valid && run_end) {
        atomicAdd(&sg[3 * j + 0], gjx);
        atomicAdd(&sg[3 * j + 1], gjy);
        atomicAdd(&sg[3 * j + 2], gjz);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      gix += __shfl_xor_sync(FULL, gix, o);
      giy += __shfl_xor_sync(FULL, giy, o);
      giz += __shfl_xor_sync(FULL, giz, o);
    }
    __syncwarp();
    for (int t = lane; t < na; t += 32) {
      const int j = la[t];
      add_force(acc_w, j - a0, orig, j, F, sg[3 * t], sg[3 * t + 1], sg[3 * t + 2]);
    }
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

int nbr_chunk() { return kNbrChunk; }

size_t nbr_smem_bytes(int max_mol) {
  return (size_t)(max_mol < kNbrStageMax ? max_mol : kNbrStageMax) * sizeof(float4);
}

cudaError_t nbr_set_smem(size_t bytes) {
  static size_t cur = 0;
  if (bytes <= cur) return cudaSuccess;
  cur = bytes;
  return cudaFuncSetAttribute(k_neighbors_mol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_neighbors_mol(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                          const int4* work, int n_work, int max_mol, unsigned* status, cudaStream_t s) {
  if (n_work <= 0) return;
  k_neighbors_mol<<<n_work, 32 * kNbrWarps, nbr_smem_bytes(max_mol), s>>>(g, nl, c, work, status);
}

void launch_neighbors(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                      unsigned* status, cudaStream_t s) {
  if (g.n_atoms <= 0) return;
  const int threads = 256;
  const int blocks = (int)(((long)g.n_atoms * 32 + threads - 1) / threads);
  k_neighbors<<<blocks, threads, 0, s>>>(g, nl, c, status);
}

size_t aev_fwd_smem_bytes(int cap_r, int cap_a, int warps) {
  return (size_t)warps * aev_fwd_warp_floats(cap_r, cap_a) * sizeof(float);
}

size_t aev_adj_smem_bytes(int cap_r, int cap_a, int warps, int mol_atoms_smem_max) {
  return (size_t)warps * mol_atoms_smem_max * 3 * sizeof(double) +
         (size_t)warps * adj_warp_floats(cap_r, cap_a) * sizeof(float);
}

namespace {
template <typename Shape>
void launch_aev_shape(const Geometry& g, const NeighborLists& nl, const AevConst& c, const int* row_of_int,
                      void* out, Prec prec, int warps, cudaStream_t s, bool split) {
  const int blocks = (g.n_atoms + warps - 1) / warps;
  const size_t smem = aev_fwd_smem_bytes(nl.cap_r, nl.cap_a, warps);
  switch (prec) {
    case Prec::F32:
      launch_pdl(k_aev<float, false, Shape>, blocks, warps * 32, smem, s, g, nl, c, row_of_int, (float*)out);
      break;
    case Prec::BF16:
      if (split)
        launch_pdl(k_aev<__nv_bfloat16, true, Shape>, blocks, warps * 32, smem, s, g, nl, c, row_of_int,
                   (__nv_bfloat16*)out);
      else
        launch_pdl(k_aev<__nv_bfloat16, false, Shape>, blocks, warps * 32, smem, s, g, nl, c, row_of_int,
                   (__nv_bfloat16*)out);
      break;
    case Prec::F16:
      if (split)
        launch_pdl(k_aev<__half, true, Shape>, blocks, warps * 32, smem, s, g, nl, c, row_of_int,
                   (__half*)out);
      else
        launch_pdl(k_aev<__half, false, Shape>, blocks, warps * 32, smem, s, g, nl, c, row_of_int,
                   (__half*)out);
      break;
  }
}
}  // namespace

void launch_aev(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                const int* row_of_int, void* out, Prec prec, int warps, cudaStream_t s, bool split) {
  if (g.n_atoms <= 0) return;
  if (c.model == 1)
    launch_aev_shape<ShapeANI1x>(g, nl, c, row_of_int, out, prec, warps, s, split);
  else
    launch_aev_shape<ShapeANI2x>(g, nl, c, row_of_int, out, prec, warps, s, split);
}

int aev_adj_stage_cap(int cap_a) { return cap_a < kAdjStage ? cap_a : kAdjStage; }

size_t aev_adj_launch_smem(int cap_r, int cap_a, int warps, int mol_atoms_smem_max) {
  const size_t main = aev_adj_smem_bytes(cap_r, aev_adj_stage_cap(cap_a), warps, mol_atoms_smem_max);
  const size_t over = aev_adj_smem_bytes(cap_r, cap_a, warps, 0);
  return main > over ? main : over;
}

int aev_adj_launches(int cap_a) { return cap_a > kAdjStage ? 2 : 1; }

void launch_aev_adjoint(const Geometry& g, const NeighborLists& nl, const AevConst& c,
                        const int* row_of_int, const float* dG, const int4* work, int n_work,
                        const int* orig, double* F, int warps, int mol_atoms_smem_max, int* ovf,
                        int ovf_ctas, cudaStream_t s) {
  if (n_work <= 0) return;
  const int stage = aev_adj_stage_cap(nl.cap_a);
  // ovf[0] was zeroed at the start of the step
  auto kern = c.model == 1 ? k_aev_adjoint<ShapeANI1x> : k_aev_adjoint<ShapeANI2x>;
  launch_pdl(kern, n_work, warps * 32, aev_adj_smem_bytes(nl.cap_r, stage, warps, mol_atoms_smem_max),
             s, g, nl, c, row_of_int, dG, work, orig, F, mol_atoms_smem_max, stage, ovf, 0);
  if (stage < nl.cap_a) {
    // as many CTAs as the SMs hold at once (ovf_ctas, from aev_adj_overflow_ctas):
    // dense systems defer most centres to this launch, and their CTAs leave at
    // once when the list is short
    kern<<<ovf_ctas, warps * 32, aev_adj_smem_bytes(nl.cap_r, nl.cap_a, warps, 0), s>>>(
        g, nl, c, row_of_int, dG, work, orig, F, 0, nl.cap_a, ovf, 1);
  }
}

int aev_adj_overflow_ctas(int cap_r, int cap_a, int warps, int model) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  const size_t smem = aev_adj_smem_bytes(cap_r, cap_a, warps, 0);
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, model == 1 ? k_aev_adjoint<ShapeANI1x> : k_aev_adjoint<ShapeANI2x>, warps * 32, smem);
  if (e != cudaSuccess || per_sm <= 0) {
    cudaGetLastError();
    per_sm = 2;
  }
  return sms * per_sm;
}

// Raises (never lowers) the dynamic shared-memory limits of the featurizer
// kernels, so handles of different sizes can coexist in one process.  Handles
// may be created, tuned and rescheduled on several host threads at once: the
// maxima and the attribute updates are serialised.
cudaError_t aev_set_smem_limits(size_t fwd_bytes, size_t adj_bytes) {
  static std::mutex mu;
  static size_t fwd_max = 0, adj_max = 0;
  std::lock_guard<std::mutex> lock(mu);
  fwd_bytes = fwd_max = fwd_bytes > fwd_max ? fwd_bytes : fwd_max;
  adj_bytes = adj_max = adj_bytes > adj_max ? adj_bytes : adj_max;
  const void* fwd[] = {(const void*)k_aev<float, false, ShapeANI2x>,
                       (const void*)k_aev<__nv_bfloat16, false, ShapeANI2x>,
                       (const void*)k_aev<__half, false, ShapeANI2x>,
                       (const void*)k_aev<__nv_bfloat16, true, ShapeANI2x>,
                       (const void*)k_aev<__half, true, ShapeANI2x>,
                       (const void*)k_aev<float, false, ShapeANI1x>,
                       (const void*)k_aev<__nv_bfloat16, false, ShapeANI1x>,
                       (const void*)k_aev<__half, false, ShapeANI1x>,
                       (const void*)k_aev<__nv_bfloat16, true, ShapeANI1x>,
                       (const void*)k_aev<__half, true, ShapeANI1x>};
  for (const void* f : fwd) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_bytes);
    if (e != cudaSuccess) return e;
  }
  for (const void* f : {(const void*)k_aev_adjoint<ShapeANI2x>, (const void*)k_aev_adjoint<ShapeANI1x>}) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nnp
