// mlp_tail_tc.cu -- the second and third hidden layers, the output layer and
// their reverse pass, fused on the tensor cores (BF16 / FP16 operands, FP32
// accumulation in tensor memory).
//
// For one 128-atom tile of one element and one ensemble member:
//   h2 = celu(W2 h1 + b2)                    (L2 forward)
//   z3 = W3 h2 + b3, y = w4 . celu(z3) + b4  (L3 forward + output layer)
//   d3 = (1/M) w4 * celu'(z3)                (start of the reverse pass)
//   d2 = (d3 W3) * celu'(h2)                 (L3 reverse)
//   d1 = (d2 W2) * celu'(h1)                 (L2 reverse, written over h1)
// Only h1 comes from HBM (TMA, once) and only y and d1 go back: h2, d3 and
// d2 live in shared memory, written by the epilogue warps directly in the
// 128B-swizzled K-major layout that the next tcgen05.mma reads as its A
// operand; every accumulator lives in tensor memory.  The weights stream
// through a 3-stage TMA ring in the order the MMAs consume them.
//
// Roles (persistent CTA per SM over the tile list):
//   warp 0, one lane: TMA producer (h1 tile, then W2, W3, W3^T, W2^T blocks);
//   warp 1, one lane: tcgen05.mma issuer, one accumulator, four phases/tile;
//   warps 2-5: epilogue of each phase (TMEM lane quarter = warp % 4).
// Waits are bounded: one that gives up sets the timeout status bit, the CTA
// stops, frees its tensor memory and returns.
#include <cstring>

#include "nnp_internal.cuh"
#include "tc_common.cuh"

namespace nnp {

namespace {

using namespace tc;

constexpr int kBK = 64;
constexpr int kRing = 3;
constexpr uint32_t kBlk = 128 * kBK * 2;     // one [128][64] 16-bit block: 16 KB
constexpr uint32_t kRingBytes = 256 * kBK * 2;  // a weight block of up to 256 rows
constexpr int kA1Blocks = 4;                 // h1 (<= 256 columns); d3 reuses it
constexpr int kA2Blocks = 3;                 // h2, then d2 (<= 192 columns)
constexpr int kEpiWarps = 8;   // two per TMEM lane quarter, each half of the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kTmemCols = 256;
constexpr size_t kSmemBytes =
    (size_t)(kA1Blocks + kA2Blocks) * kBlk + (size_t)kRing * kRingBytes + 1024 + 256 +
    (kH2Max + 2 * kH3Max + 128) * sizeof(float);

struct TailMaps {
  CUtensorMap h1;   // activations [rows][M*256], box 64 x 128
  CUtensorMap w2;   // [sum h2 rows][256], box 64 x 192
  CUtensorMap w3;   // [sum h3 rows][192], box 64 x 160
  CUtensorMap w3t;  // [sum h2 rows][160], box 64 x 192
  CUtensorMap w2t;  // [sum h1 rows][192], box 64 x 256
};
constexpr int kBoxW2 = kH2Max, kBoxW3 = kH3Max, kBoxW3T = kH2Max, kBoxW2T = kH1Max;

__device__ __forceinline__ int nblocks(int k) { return (k + kBK - 1) / kBK; }

// Streams the n_kb K-blocks of one weight matrix through the ring.
__device__ __forceinline__ bool produce_weights(const CUtensorMap* map, int row0, int n_kb,
                                                uint32_t box_rows, unsigned char* ring,
                                                uint64_t* full, uint64_t* empty, uint32_t& it,
                                                const int* abort_flag) {
  for (int kb = 0; kb < n_kb; ++kb, ++it) {
    const int s = it % kRing;
    const uint32_t use = it / kRing;
    if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) return false;
    mbar_expect_tx(&full[s], box_rows * kBK * 2);
    tma_load_2d(ring + (size_t)s * kRingBytes, map, kb * kBK, row0, &full[s]);
  }
  return true;
}

// One layer's MMAs: D[128][n] (+)= A[128][k] * B[n][k]^T, A in smem blocks at
// a_base (16 KB per 64 columns), B from the ring.
__device__ __forceinline__ bool issue_layer(uint32_t tmem, const unsigned char* a_base, int k, int n,
                                            uint32_t fmt, unsigned char* ring, uint64_t* full,
                                            uint64_t* empty, uint32_t& it, const int* abort_flag) {
  const uint32_t idesc = instr_desc(fmt, (uint32_t)n);
  const int n_kb = nblocks(k);
  for (int kb = 0; kb < n_kb; ++kb, ++it) {
    const int s = it % kRing;
    if (!mbar_wait(&full[s], (it / kRing) & 1, abort_flag)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint64_t da = smem_desc_sw128(a_base + (size_t)kb * kBlk);
    const uint64_t db = smem_desc_sw128(ring + (size_t)s * kRingBytes);
    const int ksteps = min(kBK, k - kb * kBK) / 16;
    for (int j = 0; j < ksteps; ++j)
      mma_f16(tmem, da + (uint64_t)(2 * j), db + (uint64_t)(2 * j), idesc, (kb > 0 || j > 0) ? 1u : 0u);
    mma_commit(&empty[s]);
  }
  return true;
}

__device__ __forceinline__ void st_shared_v4(unsigned char* base, uint32_t off, uint4 v) {
  *reinterpret_cast<uint4*>(base + off) = v;
}
__device__ __forceinline__ uint4 ld_shared_v4(const unsigned char* base, uint32_t off) {
  return *reinterpret_cast<const uint4*>(base + off);
}

// Row r, columns c..c+15 of an [128][K] operand in 16 KB swizzled blocks.
__device__ __forceinline__ void put16(unsigned char* blocks, int r, int c, const uint32_t (&o)[8]) {
  unsigned char* b = blocks + (size_t)(c / kBK) * kBlk;
  const int cc = c % kBK;
  st_shared_v4(b, sw128_offset(r, cc), make_uint4(o[0], o[1], o[2], o[3]));
  st_shared_v4(b, sw128_offset(r, cc + 8), make_uint4(o[4], o[5], o[6], o[7]));
}
__device__ __forceinline__ void get16(const unsigned char* blocks, int r, int c, uint32_t (&o)[8]) {
  const unsigned char* b = blocks + (size_t)(c / kBK) * kBlk;
  const int cc = c % kBK;
  const uint4 x = ld_shared_v4(b, sw128_offset(r, cc)), y = ld_shared_v4(b, sw128_offset(r, cc + 8));
  o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
  o[4] = y.x; o[5] = y.y; o[6] = y.z; o[7] = y.w;
}

template <typename T>
__device__ __forceinline__ float dcelu_from_act(float h) {  // celu'(z) = 1 + h/alpha for z <= 0
  return h > 0.f ? 1.f : fmaf(10.f, h, 1.f);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_tail(const __grid_constant__ TailMaps maps, const TailProblem* __restrict__ probs,
               const GemmTile* __restrict__ tiles, int n_tiles, int reverse,
               unsigned* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* A1 = smem;                              // h1, later d3
  unsigned char* A2 = A1 + kA1Blocks * kBlk;             // h2, later d2
  unsigned char* ring = A2 + kA2Blocks * kBlk;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + kRing * kRingBytes);
  uint64_t* empty = full + kRing;
  uint64_t* a1_full = empty + kRing;
  uint64_t* a1_free = a1_full + 1;
  uint64_t* acc_ready = a1_free + 1;
  uint64_t* epi_done = acc_ready + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(epi_done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  float* sb2 = reinterpret_cast<float*>(smem + (kA1Blocks + kA2Blocks) * kBlk + kRing * kRingBytes + 256);
  float* sb3 = sb2 + kH2Max;   // per-tile copies of b2, b3, w4
  float* sw4 = sb3 + kH3Max;
  float* ypart = sw4 + kH3Max;  // [128] second half of each row's output-layer dot

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t fmt = Pack<T>::fmt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRing; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(a1_full, 1);
    mbar_init(a1_free, 1);
    mbar_init(acc_ready, 1);
    mbar_init(epi_done, kEpiWarps);  // one arrival per epilogue warp
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++tcount) {
        const GemmTile tl = tiles[tile];
        const TailProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
        if (tcount > 0 && !mbar_wait(a1_free, (tcount - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        const int nb1 = nblocks(P.h1);
        mbar_expect_tx(a1_full, (uint32_t)nb1 * kBlk);
        for (int kb = 0; kb < nb1; ++kb)
          tma_load_2d(A1 + (size_t)kb * kBlk, &maps.h1, P.a_col0 + kb * kBK, P.row0 + tl.m0, a1_full);
        ok = produce_weights(&maps.w2, P.w2_row0, nblocks(P.h1), kBoxW2, ring, full, empty, it, abort_flag) &&
             produce_weights(&maps.w3, P.w3_row0, nblocks(P.h2), kBoxW3, ring, full, empty, it, abort_flag);
        if (ok && reverse)
          ok = produce_weights(&maps.w3t, P.w3t_row0, nblocks(P.h3), kBoxW3T, ring, full, empty, it, abort_flag) &&
               produce_weights(&maps.w2t, P.w2t_row0, nblocks(P.h2), kBoxW2T, ring, full, empty, it, abort_flag);
      }
      if (!ok) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      uint32_t it = 0, tcount = 0, u_epi = 0;
      bool ok = true;
      auto wait_epi = [&]() {
        if (ok && !mbar_wait(epi_done, u_epi & 1, abort_flag)) ok = false;
        ++u_epi;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      };
      for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++tcount) {
        const GemmTile tl = tiles[tile];
        const TailProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
        if (!mbar_wait(a1_full, tcount & 1, abort_flag)) {
          ok = false;
          break;
        }
        if (tcount > 0) wait_epi();  // previous tile's last epilogue: TMEM free
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ok = ok && issue_layer(tmem, A1, P.h1, P.h2, fmt, ring, full, empty, it, abort_flag);
        if (!ok) break;
        mma_commit(acc_ready);  // L2 forward
        wait_epi();             // h2 in A2
        ok = ok && issue_layer(tmem, A2, P.h2, P.h3, fmt, ring, full, empty, it, abort_flag);
        if (!ok) break;
        mma_commit(acc_ready);  // L3 forward
        if (!reverse) {
          mma_commit(a1_free);
          continue;
        }
        wait_epi();  // d3 in A1
        ok = ok && issue_layer(tmem, A1, P.h3, P.h2, fmt, ring, full, empty, it, abort_flag);
        if (!ok) break;
        mma_commit(acc_ready);  // L3 reverse
        mma_commit(a1_free);
        wait_epi();  // d2 in A2
        ok = ok && issue_layer(tmem, A2, P.h2, P.h1, fmt, ring, full, empty, it, abort_flag);
        if (!ok) break;
        mma_commit(acc_ready);  // L2 reverse
      }
      if (!ok) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
      }
    }
  } else {
    // ---- epilogue warps 2..9: TMEM lane quarter = warp % 4, column half ----
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int et = threadIdx.x - 64;  // 0..255 over the epilogue warps
    const int r = quarter * 32 + lane;  // tile row = TMEM lane
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t u_acc = 0;
    bool ok = true;
    auto wait_acc = [&]() -> bool {
      if (ok && !mbar_wait(acc_ready, u_acc & 1, abort_flag)) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);  // the warp's tcgen05.ld calls stay converged
      ++u_acc;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      return ok;
    };
    auto done = [&]() {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // smem writes -> tensor cores
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(epi_done);
    };
    auto epi_sync = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory"); };
    // barrier of the epilogue warps that also agrees on stopping: true if any
    // of them failed a wait or another role aborted (no warp ever leaves the
    // tile loop between two barriers, so none is left waiting at one)
    auto epi_stop = [&]() -> bool {
      const int in = (!ok || *(volatile int*)abort_flag) ? 1 : 0;
      int res;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
          "bar.red.or.pred q, 1, %2, p;\n\tselp.b32 %0, 1, 0, q;\n\t}\n"
          : "=r"(res)
          : "r"(in), "r"(32 * kEpiWarps)
          : "memory");
      return res != 0;
    };
    // the two warps of a quarter (named barriers 2..5, 64 threads)
    auto pair_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(2 + quarter) : "memory"); };
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const GemmTile tl = tiles[tile];
      const TailProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
      const int row = tl.m0 + r;
      const bool row_ok = row < P.Me;
      if (epi_stop()) break;  // also: previous tile's readers of sb2/sb3/sw4/ypart are done
      for (int i = et; i < P.h2; i += 32 * kEpiWarps) sb2[i] = P.b2[i];
      for (int i = et; i < P.h3; i += 32 * kEpiWarps) {
        sb3[i] = P.b3[i];
        sw4[i] = P.w4[i];
      }
      epi_sync();

      // L2 forward: h2 = celu(acc + b2) -> A2
      {
        const int n2 = P.h2 >> 1, c0 = half * n2;
        wait_acc();
        for (int c = c0; ok && c < c0 + n2; c += 16) {
          float v[16];
          tmem_ld16(tbase + (uint32_t)c, v);
          uint32_t o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            o[i] = Pack<T>::two(celu01_fast(v[2 * i] + sb2[c + 2 * i]),
                                celu01_fast(v[2 * i + 1] + sb2[c + 2 * i + 1]));
          put16(A2, r, c, o);
        }
        done();
      }

      // L3 forward + output layer: y, d3 -> A1
      {
        const int n3 = P.h3 >> 1, c0 = half * n3;
        wait_acc();
        float yacc = 0.f;
        for (int c = c0; ok && c < c0 + n3; c += 16) {
          float v[16];
          tmem_ld16(tbase + (uint32_t)c, v);
          uint32_t o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            float dv[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int cc = c + 2 * i + h;
              const float z = v[2 * i + h] + sb3[cc];
              const float ex = expf(fminf(z, 0.f) * 10.f);  // exp(z / alpha), alpha = 0.1
              const float act = z > 0.f ? z : 0.1f * (ex - 1.f);
              const float w = sw4[cc];
              yacc = fmaf(w, act, yacc);
              dv[h] = w * (z > 0.f ? 1.f : ex) * P.inv_m;
            }
            o[i] = Pack<T>::two(dv[0], dv[1]);
          }
          if (reverse) put16(A1, r, c, o);
        }
        if (half) ypart[r] = yacc;
        pair_sync();
        if (ok && !half && row_ok) P.y[(size_t)row * P.ldy] = yacc + ypart[r] + P.b4;
        done();
      }
      if (!reverse) continue;

      // L3 reverse: d2 = acc * celu'(h2), in place in A2
      {
        const int n2 = P.h2 >> 1, c0 = half * n2;
        wait_acc();
        for (int c = c0; ok && c < c0 + n2; c += 16) {
          float v[16];
          tmem_ld16(tbase + (uint32_t)c, v);
          uint32_t hin[8], o[8];
          get16(A2, r, c, hin);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            o[i] = Pack<T>::two(v[2 * i] * dcelu_from_act<T>(Pack<T>::lo(hin[i])),
                                v[2 * i + 1] * dcelu_from_act<T>(Pack<T>::hi(hin[i])));
          put16(A2, r, c, o);
        }
        done();
      }

      // L2 reverse: d1 = acc * celu'(h1) -> global, over h1 (h1 prefetched
      // before the wait, while the last MMAs run)
      {
        const int n1 = P.h1 >> 1, c0 = half * n1;  // <= 128 columns: 8 chunks
        T* hrow = static_cast<T*>(P.h1g) + (size_t)row * P.ldh1;
        uint4 hv[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = c0 + 16 * i;
          if (row_ok && c < c0 + n1) {
            const uint4* src = reinterpret_cast<const uint4*>(hrow + c);
            hv[2 * i] = src[0];
            hv[2 * i + 1] = src[1];
          }
        }
        wait_acc();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = c0 + 16 * i;
          if (!ok || c >= c0 + n1) break;
          float v[16];
          tmem_ld16(tbase + (uint32_t)c, v);
          if (!row_ok) continue;
          const uint32_t hin[8] = {hv[2 * i].x, hv[2 * i].y, hv[2 * i].z, hv[2 * i].w,
                                   hv[2 * i + 1].x, hv[2 * i + 1].y, hv[2 * i + 1].z, hv[2 * i + 1].w};
          uint32_t o[8];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            o[k] = Pack<T>::two(v[2 * k] * dcelu_from_act<T>(Pack<T>::lo(hin[k])),
                                v[2 * k + 1] * dcelu_from_act<T>(Pack<T>::hi(hin[k])));
          uint4* dst = reinterpret_cast<uint4*>(hrow + c);
          dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
          dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
        done();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)kTmemCols));
  }
}

}  // namespace

size_t tail_maps_bytes() { return sizeof(TailMaps); }

// Row counts of the weight maps' boxes, in map order w2, w3, w3t, w2t.
int tail_weight_box(int which) {
  const int b[4] = {kBoxW2, kBoxW3, kBoxW3T, kBoxW2T};
  return b[which];
}

cudaError_t tail_set_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_tail<__nv_bfloat16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_mlp_tail<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSmemBytes);
}

// maps: HOST pointer to the five TMA descriptors (h1, w2, w3, w3t, w2t).
void launch_mlp_tail(const TailProblem* probs, const GemmTile* tiles, int n_tiles, Prec p,
                     const void* maps, int reverse, unsigned* status, cudaStream_t s) {
  if (n_tiles <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  TailMaps m;
  std::memcpy(&m, maps, sizeof(m));
  const int grid = n_tiles < sms ? n_tiles : sms;
  if (p == Prec::BF16)
    k_mlp_tail<__nv_bfloat16><<<grid, kThreads, kSmemBytes, s>>>(m, probs, tiles, n_tiles, reverse, status);
  else
    k_mlp_tail<__half><<<grid, kThreads, kSmemBytes, s>>>(m, probs, tiles, n_tiles, reverse, status);
}

}  // namespace nnp
