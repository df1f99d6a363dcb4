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
// Only h1 comes from HBM (TMA; phase 4 reads it again) and only y and d1 go
// back: h2, d3 and d2 live in shared memory, written by the epilogue warps
// directly in the 128B-swizzled K-major layout that the next tcgen05.mma
// reads as its A operand; every accumulator lives in tensor memory.  The
// weights stream through a 3-stage TMA ring in the order the MMAs consume
// them.
//
// Roles (persistent CTA per SM over the tile list):
//   warp 0, one lane: TMA producer (h1 and W2 block by block, each h1 block
//     as soon as the previous tile's MMAs are done with that block of A1;
//     then the W3, W3^T, W2^T blocks);
//   warp 18, one lane: TMA loads of phase 4's staged h1 tile;
//   warp 1: tcgen05.mma issuer (the whole warp walks the loop, an elected
//     lane issues each instruction); the four phases of a tile alternate
//     between two 256-column accumulators, and K block b of a phase waits
//     only until the epilogue has written block b of its A operand, so a
//     phase's MMAs overlap the previous phase's epilogue;
//   warps 2-17: epilogue, 64 columns at a time (TMEM lane quarter = warp % 4,
//     16 columns per warp), signalling each finished block.
// Split mode (reverse = 2, or 3 without the reverse pass; split-operand
// forward products): the first layer stored h1 as hi and lo 16-bit halves;
// the producer loads h1_hi into A1 and h1_lo into the second buffer and the
// block after it by TMA (h1_lo once the previous tile is done there: its d1
// store has read the staging memory, or without the reverse pass its last
// product has read h2_lo).  Each forward layer is three products: for layer
// 2 the two on h1_hi first (they need only A1, so they overlap the previous
// tile's last epilogue), then h1_lo x W2_hi; for layer 3 the three of each
// 64-column block as soon as phase 1's epilogue has written it (h2 as hi
// into A1 and lo into A2); phase 2's output layer then writes d3 over h2_lo.
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
constexpr int kA1Blocks = 4;                 // h1 (<= 256 columns), then h2 and d2 over it
constexpr int kA2Blocks = 3;                 // d3 (<= 160 columns); in split mode h1_lo, h2_lo first
constexpr int kEpiWarps = 16;  // four per TMEM lane quarter, 16 of every 64 columns each
constexpr int kThreads = 64 + 32 * kEpiWarps + 32;  // + the phase-4 staging loader
constexpr int kTmemCols = 512;  // two accumulators of 256 columns
// Phase 4 stages h1 in and d1 out through [kP4Boxes][128 rows][32 cols] boxes
// (64-byte swizzle) over A2 and the 16 KB after it.
constexpr uint32_t kP4Box = 128 * 32 * 2;
constexpr int kP4Boxes = kH1Max / 32;
static_assert((size_t)kP4Boxes * kP4Box <= (size_t)(kA2Blocks + 1) * kBlk, "phase-4 staging");
static_assert(kA1Blocks <= kA2Blocks + 1, "split mode: h1_lo over the second buffer and the block after it");
constexpr size_t kSmemBytes = (size_t)(kA1Blocks + kA2Blocks + 1) * kBlk + (size_t)kRing * kRingBytes +
                              1024 + 256 + 3 * 128 * sizeof(float);

struct TailMaps {
  CUtensorMap h1;   // activations [rows][M*256], box 64 x 128
  CUtensorMap w2;   // [sum h2 rows][256], box 64 x 192
  CUtensorMap w3;   // [sum h3 rows][192], box 64 x 160
  CUtensorMap w3t;  // [sum h2 rows][160], box 64 x 192
  CUtensorMap w2t;  // [sum h1 rows][192], box 64 x 256
  CUtensorMap h1s;  // activations again, box 32 x 128, 64-byte swizzle (phase 4 in and out)
};
constexpr int kBoxW2 = kH2Max, kBoxW3 = kH3Max, kBoxW3T = kH2Max, kBoxW2T = kH1Max;

__device__ __forceinline__ int nblocks(int k) { return (k + kBK - 1) / kBK; }

// Streams the n_kb K-blocks of one weight matrix (from column col0: the lo
// half of a split matrix) through the ring.
__device__ __forceinline__ bool produce_weights(const CUtensorMap* map, int row0, int n_kb,
                                                uint32_t box_rows, unsigned char* ring,
                                                uint64_t* full, uint64_t* empty, uint32_t& it,
                                                const int* abort_flag, int col0 = 0) {
  for (int kb = 0; kb < n_kb; ++kb, ++it) {
    const int s = it % kRing;
    const uint32_t use = it / kRing;
    if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) return false;
    mbar_expect_tx(&full[s], box_rows * kBK * 2);
    tma_load_2d(ring + (size_t)s * kRingBytes, map, col0 + kb * kBK, row0, &full[s]);
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

// d * celu'(z) for two values, celu'(z) from h = celu(z), alpha = 0.1:
// 1 + h / alpha for z <= 0, where it is at most 1, and 1 for z > 0, where
// 1 + h / alpha exceeds 1 (packed FP32 arithmetic).
__device__ __forceinline__ float2 times_dcelu(float2 d, float2 h) {
  const float2 g = __ffma2_rn(f2(10.f), h, f2(1.f));
  return __fmul2_rn(d, make_float2(fminf(g.x, 1.f), fminf(g.y, 1.f)));
}

// Row r, columns c..c+15 (c a multiple of 16) of the phase-4 tile: box c / 32,
// 64-byte rows whose 16-byte chunk k sits at position k ^ ((r / 2) % 4), the
// layout of a TMA box with 64-byte swizzle.
__device__ __forceinline__ uint32_t p4_offset(int r, int c) {
  return (uint32_t)(c >> 5) * kP4Box + (uint32_t)(r * 64);
}
__device__ __forceinline__ uint32_t p4_chunk(int r, int k) { return (uint32_t)(((k ^ (r >> 1)) & 3) << 4); }
__device__ __forceinline__ void get16_p4(const unsigned char* p4, int r, int c, uint32_t (&o)[8]) {
  const unsigned char* b = p4 + p4_offset(r, c);
  const int k = (c & 31) >> 3;
  const uint4 x = ld_shared_v4(b, p4_chunk(r, k)), y = ld_shared_v4(b, p4_chunk(r, k + 1));
  o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
  o[4] = y.x; o[5] = y.y; o[6] = y.z; o[7] = y.w;
}
__device__ __forceinline__ void put16_p4(unsigned char* p4, int r, int c, const uint32_t (&o)[8]) {
  unsigned char* b = p4 + p4_offset(r, c);
  const int k = (c & 31) >> 3;
  st_shared_v4(b, p4_chunk(r, k), make_uint4(o[0], o[1], o[2], o[3]));
  st_shared_v4(b, p4_chunk(r, k + 1), make_uint4(o[4], o[5], o[6], o[7]));
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_tail(const __grid_constant__ TailMaps maps, const TailProblem* __restrict__ probs,
               const GemmTile* __restrict__ tiles, const int* __restrict__ cta_off, int reverse,
               unsigned* __restrict__ status, const int* __restrict__ abort_req) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // rounded up to 1024 bytes by pointer arithmetic, so that accesses through
  // it stay shared-memory accesses
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* A1 = smem;                              // h1, then h2, then d2 in place
  unsigned char* A2 = A1 + kA1Blocks * kBlk;             // d3
  unsigned char* P4 = A2;  // phase 4: h1 in, d1 out, over A2 and the next 16 KB
  unsigned char* ring = A2 + (kA2Blocks + 1) * kBlk;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + kRing * kRingBytes);
  uint64_t* empty = full + kRing;
  uint64_t* a1_full = empty + kRing;  // [4] producer -> MMA: block b of h1 loaded
  uint64_t* a1_free = a1_full + 4;    // [4] MMA -> producer: block b of A1 consumed
  uint64_t* acc_ready = a1_free + 4;  // [2] MMA -> epilogue, per accumulator
  uint64_t* acc_free = acc_ready + 2;  // [2] epilogue -> MMA: accumulator drained
  uint64_t* blk_done = acc_free + 2;   // [4] epilogue -> MMA: 64-column block of the next A written
  uint64_t* p4_full = blk_done + 4;    // producer -> epilogue: the tile's h1 is in P4
  uint64_t* a2_free = p4_full + 1;     // MMA -> P4 loader: phase-3 MMAs are done with d3 (A2)
  uint64_t* lo_full = a2_free + 1;     // [4] split mode: producer -> MMA, block b of h1_lo loaded
  uint64_t* p4_drained = lo_full + kA1Blocks;  // split mode: epilogue -> producer, d1 store read P4
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(p4_drained + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  // [3][128]: the output-layer dot of each row over the column groups 1-3
  float* ypart = reinterpret_cast<float*>(ring + kRing * kRingBytes + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t fmt = Pack<T>::fmt;
  const bool split = reverse >= 2;                     // the tile starts at layer 3
  const bool with_rev = reverse == 1 || reverse == 2;  // the reverse phases run
  const int tile_begin = cta_off[blockIdx.x], tile_end = cta_off[blockIdx.x + 1];  // this CTA's tiles

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRing; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kA1Blocks; ++b) {
      mbar_init(&a1_full[b], 1);
      mbar_init(&a1_free[b], 1);
    }
    for (int x = 0; x < 2; ++x) {
      mbar_init(&acc_ready[x], 1);
      mbar_init(&acc_free[x], kEpiWarps);
    }
    for (int b = 0; b < 4; ++b) mbar_init(&blk_done[b], kEpiWarps);
    mbar_init(p4_full, 1);
    mbar_init(a2_free, 1);
    for (int b = 0; b < kA1Blocks; ++b) mbar_init(&lo_full[b], 1);
    mbar_init(p4_drained, 1);
    *abort_flag = *abort_req;  // nonzero only in tests of the abort path
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
  // prologue done: the next kernel may launch; h1 comes from the kernel before
  pdl_launch_dependents();
  pdl_wait();

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      uint32_t it = 0, tcount = 0;
      int first = 0;  // first A1 block the previous tile freed (past its h2 blocks)
      // an abort requested at the start: nothing is loaded (the other roles'
      // first waits give up on the flag)
      bool ok = *(volatile int*)abort_flag == 0;
      for (int tile = tile_begin; ok && tile < tile_end; ++tile, ++tcount) {
        const GemmTile tl = tiles[tile];
        const TailProblem P = probs[tl.problem];
        if (split) {
          const int nb1 = nblocks(P.h1), nb2 = nblocks(P.h2);
          // h1_hi into A1 as the previous tile frees each block (blocks past
          // h1 get a plain arrival: every block completes once a tile)
          for (int kb = 0; ok && kb < kA1Blocks; ++kb) {
            if (tcount > 0 && !mbar_wait(&a1_free[kb], (tcount - 1) & 1, abort_flag)) {
              ok = false;
              break;
            }
            if (kb >= nb1) {
              mbar_arrive(&a1_full[kb]);
              continue;
            }
            mbar_expect_tx(&a1_full[kb], kBlk);
            tma_load_2d(A1 + (size_t)kb * kBlk, &maps.h1, P.a_col0 + kb * kBK, P.row0 + tl.m0, &a1_full[kb]);
          }
          // W2_hi and W2_lo for the two products on h1_hi, which need nothing else
          ok = ok &&
               produce_weights(&maps.w2, P.w2_row0, nb1, kBoxW2, ring, full, empty, it, abort_flag) &&
               produce_weights(&maps.w2, P.w2_row0, nb1, kBoxW2, ring, full, empty, it, abort_flag, kH1Max);
          // h1_lo into the second buffer and the block after it (four blocks)
          // once the previous tile is done there: its d1 store has read P4,
          // or (without the reverse pass) its last product has read h2_lo
          if (ok && tcount > 0 && !mbar_wait(with_rev ? p4_drained : a2_free, (tcount - 1) & 1, abort_flag))
            ok = false;
          for (int kb = 0; ok && kb < kA1Blocks; ++kb) {
            if (kb >= nb1) {
              mbar_arrive(&lo_full[kb]);
              continue;
            }
            mbar_expect_tx(&lo_full[kb], kBlk);
            tma_load_2d(A2 + (size_t)kb * kBlk, &maps.h1, P.h1_lo + P.a_col0 + kb * kBK, P.row0 + tl.m0,
                        &lo_full[kb]);
          }
          ok = ok && produce_weights(&maps.w2, P.w2_row0, nb1, kBoxW2, ring, full, empty, it, abort_flag);
          // W3 block by block, in the order of layer 3's products: hi, lo, hi
          for (int kb = 0; ok && kb < nb2; ++kb)
            ok = produce_weights(&maps.w3, P.w3_row0, 1, kBoxW3, ring, full, empty, it, abort_flag, kb * kBK) &&
                 produce_weights(&maps.w3, P.w3_row0, 1, kBoxW3, ring, full, empty, it, abort_flag,
                                 kH2Max + kb * kBK) &&
                 produce_weights(&maps.w3, P.w3_row0, 1, kBoxW3, ring, full, empty, it, abort_flag, kb * kBK);
          if (ok && with_rev)
            ok = produce_weights(&maps.w3t, P.w3t_row0, nblocks(P.h3), kBoxW3T, ring, full, empty, it, abort_flag) &&
                 produce_weights(&maps.w2t, P.w2t_row0, nb2, kBoxW2T, ring, full, empty, it, abort_flag);
          continue;
        }
        const int nb1 = nblocks(P.h1);
        // h1 and the matching W2 block, block by block, each as soon as the
        // previous tile is done with that block of A1 (the blocks it freed
        // first, first); blocks past h1 get a plain arrival
        for (int i = 0; ok && i < kA1Blocks; ++i) {
          const int kb = (first + i) % kA1Blocks;
          if (tcount > 0 && !mbar_wait(&a1_free[kb], (tcount - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          if (kb >= nb1) {
            mbar_arrive(&a1_full[kb]);
            continue;
          }
          mbar_expect_tx(&a1_full[kb], kBlk);
          tma_load_2d(A1 + (size_t)kb * kBlk, &maps.h1, P.a_col0 + kb * kBK, P.row0 + tl.m0, &a1_full[kb]);
          const int s = it % kRing;
          const uint32_t use = it / kRing;
          if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], kBoxW2 * kBK * 2);
          tma_load_2d(ring + (size_t)s * kRingBytes, &maps.w2, kb * kBK, P.w2_row0, &full[s]);
          ++it;
        }
        first = nblocks(P.h2);
        ok = ok && produce_weights(&maps.w3, P.w3_row0, nblocks(P.h2), kBoxW3, ring, full, empty, it, abort_flag);
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
    {
      // ---- MMA issuer: phases alternate between the two accumulators; a
      // phase's K block b waits only for block b of its A operand.  The whole
      // warp walks the loop (its values stay warp-uniform) and one elected
      // lane issues each tcgen05 instruction ----
      uint32_t it = 0, tcount = 0;
      uint32_t used[2] = {0, 0};       // phases issued per accumulator
      uint32_t blk_waits[4] = {0, 0, 0, 0};
      bool ok = true;
      // phases 2-4: K block b waits for block b of the A operand from the
      // epilogue; blk_free: commit each K block's completion there (the
      // last reader of that block of A1)
      // split mode: waits for the TMA loads of h1_hi (A1) and h1_lo
      uint32_t a1_waits[kA1Blocks] = {0, 0, 0, 0};
      uint32_t lo_waits[kA1Blocks] = {0, 0, 0, 0};
      // a_ready / a_waits: the barriers (and the waits so far) that block b of
      // the A operand completes (the epilogue's blk_done)
      auto phase = [&](int x, const unsigned char* a_base, int k, int n, uint64_t* blk_free,
                       uint64_t* a_ready, uint32_t* a_waits) {
        if (!ok) return;
        if (used[x] > 0 && !mbar_wait_warp(&acc_free[x], (used[x] - 1) & 1, abort_flag)) {
          ok = false;
          return;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = instr_desc(fmt, (uint32_t)n);
        const uint32_t d = tmem + (uint32_t)(x * kTmemCols / 2);
        const int n_kb = nblocks(k);
        for (int kb = 0; kb < n_kb; ++kb, ++it) {
          if (!mbar_wait_warp(&a_ready[kb], a_waits[kb] & 1, abort_flag)) {
            ok = false;
            return;
          }
          ++a_waits[kb];
          const int s = it % kRing;
          if (!mbar_wait_warp(&full[s], (it / kRing) & 1, abort_flag)) {
            ok = false;
            return;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da = smem_desc_sw128(a_base + (size_t)kb * kBlk);
          const uint64_t db = smem_desc_sw128(ring + (size_t)s * kRingBytes);
          const int ksteps = min(kBK, k - kb * kBK) / 16;
          if (ksteps == 4) {
            mma_f16_elect4(d, da, db, idesc, kb > 0 ? 1u : 0u);
          } else {
            for (int j = 0; j < ksteps; ++j)
              mma_f16_elect(d, da + (uint64_t)(2 * j), db + (uint64_t)(2 * j), idesc, (kb > 0 || j > 0) ? 1u : 0u);
          }
          mma_commit_elect(&empty[s]);
          if (blk_free) mma_commit_elect(&blk_free[kb]);
        }
        mma_commit_elect(&acc_ready[x]);
        ++used[x];
      };
      // L2 forward: A = h1, taken block by block in the order the producer
      // loads it (the blocks the previous tile freed first, first)
      auto phase1 = [&](const TailProblem& P, int first) {
        if (!ok) return;
        if (used[0] > 0 && !mbar_wait_warp(&acc_free[0], (used[0] - 1) & 1, abort_flag)) {
          ok = false;
          return;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = instr_desc(fmt, (uint32_t)P.h2);
        const uint32_t d = tmem;
        const int nb1 = nblocks(P.h1);
        bool acc = false;
        for (int i = 0; i < kA1Blocks; ++i) {
          const int kb = (first + i) % kA1Blocks;
          if (!mbar_wait_warp(&a1_full[kb], tcount & 1, abort_flag)) {
            ok = false;
            return;
          }
          if (kb >= nb1) continue;
          const int s = it % kRing;
          if (!mbar_wait_warp(&full[s], (it / kRing) & 1, abort_flag)) {
            ok = false;
            return;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da = smem_desc_sw128(A1 + (size_t)kb * kBlk);
          const uint64_t db = smem_desc_sw128(ring + (size_t)s * kRingBytes);
          const int ksteps = min(kBK, P.h1 - kb * kBK) / 16;
          if (ksteps == 4) {
            mma_f16_elect4(d, da, db, idesc, acc ? 1u : 0u);
            acc = true;
          } else {
            for (int j = 0; j < ksteps; ++j) {
              mma_f16_elect(d, da + (uint64_t)(2 * j), db + (uint64_t)(2 * j), idesc, acc ? 1u : 0u);
              acc = true;
            }
          }
          mma_commit_elect(&empty[s]);
          ++it;
        }
        mma_commit_elect(&acc_ready[0]);
        ++used[0];
        // A1 blocks past h2 are not read again in this tile
        for (int kb = nblocks(P.h2); kb < kA1Blocks; ++kb) mma_commit_elect(&a1_free[kb]);
      };
      // split mode, a forward layer (K = k, N = n) as three products in the
      // producer's ring order: A_hi B_hi and A_hi B_lo (A_hi in A1), then
      // A_lo B_hi (A_lo in the second buffer), each over all K blocks; or,
      // with by_block, the three products of K block b as soon as block b is
      // ready (A_hi and A_lo of a block announced together on hi_ready).
      // Before its first use, K block b of A_hi waits on hi_ready[b] and of
      // A_lo on lo_ready[b] (null: no wait), for b < n_wait (blocks past k
      // complete their barrier but issue nothing); after the A_hi products, A1
      // blocks from keep_a1 on are free.
      auto phase_split = [&](int x, int k, int n, int n_wait, uint64_t* hi_ready, uint32_t* hi_waits,
                             uint64_t* lo_ready, uint32_t* lo_waits, int keep_a1, bool by_block) {
        if (!ok) return;
        if (used[x] > 0 && !mbar_wait_warp(&acc_free[x], (used[x] - 1) & 1, abort_flag)) {
          ok = false;
          return;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = instr_desc(fmt, (uint32_t)n);
        const uint32_t d = tmem + (uint32_t)(x * kTmemCols / 2);
        const int n_kb = nblocks(k);
        bool acc = false;
        auto wait_ready = [&](uint64_t* ready, uint32_t* waits, int kb) -> bool {
          if (!ready) return true;
          if (!mbar_wait_warp(&ready[kb], waits[kb] & 1, abort_flag)) return false;
          ++waits[kb];
          return true;
        };
        // one ring block: K block kb of A_hi (A1) or A_lo (second buffer)
        auto issue = [&](bool lo_half, int kb) -> bool {
          const int s = it % kRing;
          if (!mbar_wait_warp(&full[s], (it / kRing) & 1, abort_flag)) return false;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da = smem_desc_sw128((lo_half ? A2 : A1) + (size_t)kb * kBlk);
          const uint64_t db = smem_desc_sw128(ring + (size_t)s * kRingBytes);
          const int ksteps = min(kBK, k - kb * kBK) / 16;
          if (ksteps == 4) {
            mma_f16_elect4(d, da, db, idesc, acc ? 1u : 0u);
            acc = true;
          } else {
            for (int j = 0; j < ksteps; ++j) {
              mma_f16_elect(d, da + (uint64_t)(2 * j), db + (uint64_t)(2 * j), idesc, acc ? 1u : 0u);
              acc = true;
            }
          }
          mma_commit_elect(&empty[s]);
          ++it;
          return true;
        };
        if (by_block) {
          for (int kb = 0; kb < n_kb; ++kb)
            if (!wait_ready(hi_ready, hi_waits, kb) || !issue(false, kb) || !issue(false, kb) || !issue(true, kb)) {
              ok = false;
              return;
            }
        } else {
          for (int seg = 0; seg < 3; ++seg) {
            uint64_t* ready = seg == 0 ? hi_ready : seg == 2 ? lo_ready : nullptr;
            uint32_t* waits = seg == 0 ? hi_waits : lo_waits;
            for (int kb = 0; kb < (ready ? n_wait : n_kb); ++kb)
              if (!wait_ready(ready, waits, kb) || (kb < n_kb && !issue(seg == 2, kb))) {
                ok = false;
                return;
              }
            if (seg == 1)
              for (int kb = keep_a1; kb < kA1Blocks; ++kb) mma_commit_elect(&a1_free[kb]);
          }
        }
        mma_commit_elect(&acc_ready[x]);
        ++used[x];
      };
      int first = 0;
      for (int tile = tile_begin; ok && tile < tile_end; ++tile, ++tcount) {
        const GemmTile tl = tiles[tile];
        const TailProblem P = probs[tl.problem];
        if (split) {
          const int nb2 = nblocks(P.h2);
          // L2 forward: h1_hi (A1) and h1_lo (second buffer) loaded by TMA;
          // A1 blocks past h2 are free after the products on h1_hi
          phase_split(0, P.h1, P.h2, kA1Blocks, a1_full, a1_waits, lo_full, lo_waits, nb2, false);
          // L3 forward: h2_hi (A1) and h2_lo (A2) from the epilogue, block b
          // of both announced by one blk_done arrival, its three products
          // issued as soon as it is written
          phase_split(1, P.h2, P.h3, nb2, blk_done, blk_waits, nullptr, nullptr, kA1Blocks, true);
          if (!with_rev) {  // the last readers of A1 and A2 in this tile
            for (int kb = 0; ok && kb < nb2; ++kb) mma_commit_elect(&a1_free[kb]);
            if (ok) mma_commit_elect(a2_free);
            continue;
          }
          phase(0, A2, P.h3, P.h2, nullptr, blk_done, blk_waits);  // L3 reverse, block by block of d3
          if (ok) mma_commit_elect(a2_free);                      // A2 may take phase 4's h1
          phase(1, A1, P.h2, P.h1, a1_free, blk_done, blk_waits);  // L2 reverse, d2 over h2_hi
          continue;
        }
        phase1(P, first);                 // L2 forward
        first = nblocks(P.h2);
        // L3 forward, block by block of h2 (over h1); without the reverse
        // pass it is the last reader of those blocks of A1
        phase(1, A1, P.h2, P.h3, reverse ? nullptr : a1_free, blk_done, blk_waits);
        if (!reverse) continue;
        phase(0, A2, P.h3, P.h2, nullptr, blk_done, blk_waits);  // L3 reverse, block by block of d3
        if (ok) mma_commit_elect(a2_free);        // d3 consumed: A2 may take phase 4's h1
        phase(1, A1, P.h2, P.h1, a1_free, blk_done, blk_waits);  // L2 reverse, block by block of d2 (over h2)
      }
      if (!ok && lane == 0) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
      }
    }
  } else if (warp == 2 + kEpiWarps) {
    if (lane == 0 && with_rev) {
      // ---- phase-4 staging loader: h1 of each tile into P4 once the tile's
      // phase-3 MMAs are done with d3 in A2 (apart from the ring producer,
      // whose next weights must not wait for that) ----
      uint32_t k = 0;
      bool ok = true;
      for (int tile = tile_begin; tile < tile_end; ++tile, ++k) {
        const GemmTile tl = tiles[tile];
        const TailProblem P = probs[tl.problem];
        if (!mbar_wait(a2_free, k & 1, abort_flag)) {
          ok = false;
          break;
        }
        const int nbox = P.h1 / 32;
        mbar_expect_tx(p4_full, (uint32_t)nbox * kP4Box);
        for (int j = 0; j < nbox; ++j)
          tma_load_2d(P4 + (size_t)j * kP4Box, &maps.h1s, P.a_col0 + 32 * j, P.row0 + tl.m0, p4_full);
      }
      if (!ok) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
      }
    }
  } else {
    // ---- epilogue warps 2..17: TMEM lane quarter = warp % 4, column group ----
    const int quarter = warp & 3, grp = (warp - 2) >> 2;
    const int et = threadIdx.x - 64;  // 0..255 over the epilogue warps
    const int r = quarter * 32 + lane;  // tile row = TMEM lane
    const uint32_t tq = (uint32_t)(quarter * 32) << 16;
    uint32_t ready_waits[2] = {0, 0}, p4_waits = 0;
    bool ok = true;
    auto wait_acc = [&](int x) -> uint32_t {  // TMEM address of accumulator x for this warp
      if (ok && !mbar_wait(&acc_ready[x], ready_waits[x] & 1, abort_flag)) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);  // the warp's tcgen05.ld calls stay converged
      ++ready_waits[x];
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      return tmem + (uint32_t)(x * kTmemCols / 2) + tq;
    };
    // block b of the next A operand written: publish it to the tensor cores
    auto arrive = [&](uint64_t* bar) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar);
    };
    // accumulator drained: order the TMEM loads before the next MMA into it
    // (no shared-memory hand-off, hence no proxy fence, which would also wait
    // for this warp's global stores)
    auto release = [&](uint64_t* bar) {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar);
    };
    auto epi_sync = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory"); };
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
    auto quad_sync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(2 + quarter) : "memory"); };
    // columns of block b handled by this warp: [b*64 + grp*16, ... + 16) if below n
    auto my_cols = [&](int b, int n, int& c0, int& c1) {
      c0 = b * kBK + grp * 16;
      c1 = min(c0 + 16, n);
    };
    for (int tile = tile_begin; tile < tile_end; ++tile) {
      const GemmTile tl = tiles[tile];
      const TailProblem P = probs[tl.problem];
      const int row = tl.m0 + r;
      const bool row_ok = row < P.Me;
      // the barrier ends the previous tile's readers of ypart
      if (epi_stop()) break;
      {  // warm the L1 with this tile's b2, b3 and w4 (128-byte lines, one per thread)
        const int l2 = (P.h2 + 31) / 32, l3 = (P.h3 + 31) / 32;
        const float* line = et < l2 ? P.b2 + 32 * et
                            : et < l2 + l3 ? P.b3 + 32 * (et - l2)
                            : et < l2 + 2 * l3 ? P.w4 + 32 * (et - l2 - l3) : nullptr;
        if (line) asm volatile("prefetch.global.L1 [%0];" ::"l"(line));
      }

      // phase 1, L2 forward (accumulator 0): h2 = celu(acc + b2) -> A1 (its
      // MMAs, the last readers of h1 there, are complete), block by block; in
      // split mode as hi = round(h2) into A1 and lo = round(h2 - hi) into A2
      {
        const uint32_t t = wait_acc(0);
        for (int b = 0; b < nblocks(P.h2); ++b) {
          int c0, c1;
          my_cols(b, P.h2, c0, c1);
          for (int c = c0; ok && c < c1; c += 16) {
            float bias[16], v[16];
            ldg16(P.b2 + c, bias);  // in flight during the TMEM load
            tmem_ld16(t + (uint32_t)c, v);
            uint32_t o[8], lo[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float2 h, e;
              celu01_pair(__fadd2_rn(make_float2(v[2 * i], v[2 * i + 1]), make_float2(bias[2 * i], bias[2 * i + 1])),
                          h, e);
              o[i] = Pack<T>::two(h.x, h.y);
              lo[i] = Pack<T>::two(h.x - Pack<T>::lo(o[i]), h.y - Pack<T>::hi(o[i]));
            }
            put16(A1, r, c, o);
            if (split) put16(A2, r, c, lo);
          }
          arrive(&blk_done[b]);
        }
        release(&acc_free[0]);
      }

      // phase 2, L3 forward + output layer (accumulator 1): y, d3 -> A2
      {
        const uint32_t t = wait_acc(1);
        if (with_rev) {  // the previous tile's d1 store has read P4 (over A2)
          if (et == 0) bulk_wait_read();
          epi_sync();
        }
        float2 yacc2 = f2(0.f);  // even and odd columns
        for (int b = 0; b < nblocks(P.h3); ++b) {
          int c0, c1;
          my_cols(b, P.h3, c0, c1);
          for (int c = c0; ok && c < c1; c += 16) {
            float b3[16], w4[16], v[16];
            ldg16(P.b3 + c, b3);  // in flight during the TMEM load
            ldg16(P.w4 + c, w4);
            tmem_ld16(t + (uint32_t)c, v);
            uint32_t o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float2 w = make_float2(w4[2 * i], w4[2 * i + 1]);
              float2 h, ex;  // celu(z) and celu'(z)
              celu01_pair(__fadd2_rn(make_float2(v[2 * i], v[2 * i + 1]), make_float2(b3[2 * i], b3[2 * i + 1])),
                          h, ex);
              yacc2 = __ffma2_rn(w, h, yacc2);
              const float2 dv = __fmul2_rn(__fmul2_rn(w, f2(P.inv_m)), ex);
              o[i] = Pack<T>::two(dv.x, dv.y);
            }
            if (with_rev) put16(A2, r, c, o);
          }
          if (with_rev) arrive(&blk_done[b]);
        }
        const float yacc = yacc2.x + yacc2.y;
        if (grp) ypart[(grp - 1) * 128 + r] = yacc;
        quad_sync();
        if (ok && !grp && row_ok)
          P.y[(size_t)row * P.ldy] = yacc + ypart[r] + ypart[128 + r] + ypart[256 + r] + P.b4;
        release(&acc_free[1]);
      }
      if (!with_rev) continue;

      // phase 3, L3 reverse (accumulator 0): d2 = acc * celu'(h2), in place in A1
      {
        const uint32_t t = wait_acc(0);
        for (int b = 0; b < nblocks(P.h2); ++b) {
          int c0, c1;
          my_cols(b, P.h2, c0, c1);
          for (int c = c0; ok && c < c1; c += 16) {
            float v[16];
            tmem_ld16(t + (uint32_t)c, v);
            uint32_t hin[8], o[8];
            get16(A1, r, c, hin);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float2 d = times_dcelu(make_float2(v[2 * i], v[2 * i + 1]),
                                           make_float2(Pack<T>::lo(hin[i]), Pack<T>::hi(hin[i])));
              o[i] = Pack<T>::two(d.x, d.y);
            }
            put16(A1, r, c, o);
          }
          arrive(&blk_done[b]);
        }
        release(&acc_free[0]);
      }

      // phase 4, L2 reverse (accumulator 1): d1 = acc * celu'(h1), h1 staged in
      // P4 by TMA and overwritten there by d1, which one thread then stores
      // with TMA (this warp: every fourth 16-column chunk of its 32 rows)
      {
        const uint32_t t = wait_acc(1);
        if (ok && !mbar_wait(p4_full, p4_waits & 1, abort_flag)) {
          atomicOr(status, kStatTimeout);
          atomicExch(abort_flag, 1);
          ok = false;
        }
        ok = __all_sync(0xffffffffu, ok);
        ++p4_waits;
        for (int c = grp * 16; ok && c < P.h1; c += 64) {
          float v[16];
          tmem_ld16(t + (uint32_t)c, v);
          uint32_t hin[8], o[8];
          get16_p4(P4, r, c, hin);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float2 d = times_dcelu(make_float2(v[2 * k], v[2 * k + 1]),
                                         make_float2(Pack<T>::lo(hin[k]), Pack<T>::hi(hin[k])));
            o[k] = Pack<T>::two(d.x, d.y);
          }
          put16_p4(P4, r, c, o);
        }
        release(&acc_free[1]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_sync();
        if (et == 0 && ok) {
          for (int j = 0; j < P.h1 / 32; ++j)
            tma_store_2d(&maps.h1s, P4 + (size_t)j * kP4Box, P.a_col0 + 32 * j, P.row0 + tl.m0);
          bulk_commit();
          if (split) {  // the producer's next h1_lo load goes over P4
            bulk_wait_read();
            mbar_arrive(p4_drained);
          }
        }
      }
    }
    if (et == 0) bulk_wait_all();
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

// maps: HOST pointer to the TMA descriptors (h1, w2, w3, w3t, w2t, h1 in
// 32-column boxes); CTA c runs the tiles cta_off[c] .. cta_off[c + 1].
void launch_mlp_tail(const TailProblem* probs, const GemmTile* tiles, const int* cta_off, int n_ctas,
                     Prec p, const void* maps, int reverse, unsigned* status, const int* abort_req,
                     cudaStream_t s) {
  if (n_ctas <= 0) return;
  TailMaps m;
  std::memcpy(&m, maps, sizeof(m));
  if (p == Prec::BF16)
    launch_pdl(k_mlp_tail<__nv_bfloat16>, n_ctas, kThreads, kSmemBytes, s, m, probs, tiles, cta_off,
               reverse, status, abort_req);
  else
    launch_pdl(k_mlp_tail<__half>, n_ctas, kThreads, kSmemBytes, s, m, probs, tiles, cta_off,
               reverse, status, abort_req);
}

}  // namespace nnp
