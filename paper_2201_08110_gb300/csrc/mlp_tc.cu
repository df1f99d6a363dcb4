// mlp_tc.cu -- grouped matrix products of the atomic networks on the 5th-gen
// tensor cores: BF16 or FP16 operands, FP32 accumulation in tensor memory.
//
// The networks of every element and ensemble member run as one launch per
// layer (Sec. 2 "Optimization": the ensemble is evaluated in parallel over
// networks and atoms).  D = A * B^T, A and B K-major, in 128 x N output tiles
// (N <= 256, set per tile in the instruction descriptor).  The kernel is
// persistent (one CTA per SM walks the tile list) and warp-specialised:
//   * warp 0, one lane: TMA producer, 64-wide K blocks of A (128 rows) and B
//     (up to 256 rows) into a 4-stage ring of 128B-swizzled shared memory,
//     running ahead across tile boundaries;
//   * warp 1, one lane: issues tcgen05.mma (M = 128, K = 16 per instruction)
//     into one of two 256-column FP32 accumulators in tensor memory, releases
//     each stage with tcgen05.commit and signals the finished accumulator;
//   * warps 2-9: epilogue, tcgen05.ld of the rows they own (warp w reads TMEM
//     lanes 32 (w % 4) ...), bias + CELU fused (forward) or plain FP32
//     (reverse), written into a 128B-swizzled staging box in shared memory
//     that one thread stores with TMA; the two halves of the epilogue warps
//     take alternate boxes, each with its own staging buffer.
// With two accumulators the epilogue of one tile overlaps the MMAs of the
// next.  Every mbarrier wait is bounded; a wait that gives up sets the status
// word's timeout bit, every role stops, the CTA frees its tensor memory and
// returns.
#include <cuda.h>

#include <cstring>

#include "nnp_internal.cuh"
#include "tc_common.cuh"

namespace nnp {

namespace {

using namespace tc;

constexpr int kBM = 128;       // tile rows (atoms)
constexpr int kBNMax = 256;    // tile columns, TMEM columns per accumulator
constexpr int kBK = 64;        // K per stage (128 bytes of 16-bit elements)
constexpr int kStages = 4;
constexpr int kEpiWarps = 8;   // two per TMEM lane quarter, each half of the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer, MMA, epilogue warps
constexpr uint32_t kABytes = kBM * kBK * 2;      // 16 KB
constexpr uint32_t kBBytes = kBNMax * kBK * 2;   // 32 KB (room for 256 B rows)
constexpr uint32_t kStageBytes = kABytes + kBBytes;
constexpr uint32_t kStgBytes = 128 * 128;        // one output box: 128 rows x 128 bytes
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + 2 * kStgBytes + 1024 /*align*/ +
                              256 /*barriers*/;

// CTA pairs (first layer): each CTA stages its 128 rows of A and half of
// B's rows, so a stage is 32 KB and six fit.
constexpr int kStages2 = 6;
constexpr uint32_t kBHalfBytes = (kBNMax / 2) * kBK * 2;  // 16 KB
constexpr uint32_t kStageBytes2 = kABytes + kBHalfBytes;
constexpr size_t kSmemBytes2 = (size_t)kStages2 * kStageBytes2 + 2 * kStgBytes + 1024 /*align*/ + 256 /*barriers*/;

struct TcMaps {
  CUtensorMap a;
  CUtensorMap b;
  CUtensorMap d;  // output, 128-row boxes of 128 bytes (64 16-bit or 32 FP32 columns)
};
static_assert(sizeof(CUtensorMap) == 128, "tensor map slots are 128 bytes");

// Row r, FP32 columns c..c+15 (c a multiple of 16) of a [128][32] FP32 box in
// the 128-byte-swizzled layout: 16-byte chunk k of row r at k ^ (r % 8).
__device__ __forceinline__ void put16_f32(unsigned char* box, int r, int c, const float (&v)[16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = (c >> 2) + i;
    *reinterpret_cast<float4*>(box + r * 128 + ((k ^ (r & 7)) << 4)) =
        make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  }
}

// The epilogue of one output tile for the FP32 store (dE/dG) and the
// bias + CELU (16-bit, optionally split) cases: this thread's TMEM lane (tile
// row r, row `row` of the output map's first row) and this half's boxes.
template <typename T>
__device__ __forceinline__ void epi_store_tile(const GemmProblem& P, int n0, int n_tile, uint32_t tbase,
                                               unsigned char* stg, int r, int half, bool leader,
                                               bool& in_flight, const CUtensorMap* dmap, int row) {
  auto half_sync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(2 + half) : "memory"); };
  if (P.epi == (int)Epi::Store) {
    // dE/dG, FP32: 32-column boxes, one TMEM load each (columns past the
    // problem's stored as zeros)
    const int nbox = (n_tile + 31) / 32;
    for (int bx = half; bx < nbox; bx += 2) {
      if (leader && in_flight) bulk_wait_read();  // the previous store has read stg
      half_sync();
      const int c = bx * 32;
      float v[32];
      tmem_ld32(tbase + (uint32_t)c, v);  // c + 32 <= 256: inside the accumulator
#pragma unroll
      for (int i = 16; i < 32; ++i)
        if (c + 16 >= n_tile) v[i] = 0.f;
      put16_f32(stg, r, 0, *reinterpret_cast<const float(*)[16]>(v));
      put16_f32(stg, r, 16, *reinterpret_cast<const float(*)[16]>(v + 16));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      half_sync();
      if (leader) {
        tma_store_2d(dmap, stg, P.d_col0 + n0 + c, row);
        bulk_commit();
        in_flight = true;
      }
    }
  } else {
    // bias + CELU into T, 64-column boxes.  With a split output (d_lo >
    // 0) each value is computed once: hi = round(v) goes to the box, and
    // lo = round(v - hi) (exact in FP32 before its rounding) waits in
    // registers until the hi box has been read, then goes out as a second
    // box d_lo columns to the right.
    const int nbox = (n_tile + 63) / 64;
    const bool two = P.d_lo > 0;
    for (int bx = half; bx < nbox; bx += 2) {
      if (leader && in_flight) bulk_wait_read();  // the previous store has read stg
      half_sync();
      uint32_t lo[32];
#pragma unroll
      for (int h32 = 0; h32 < 2; ++h32) {
        const int c = bx * 64 + h32 * 32;  // column in the tile
        float v[32];
        if (c < n_tile) tmem_ld32(tbase + (uint32_t)c, v);  // warp-uniform; c + 32 <= 256
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int cq = c + 16 * q;
          float b[16];
          if (cq < n_tile) {  // bias only for the problem's columns (no read past it)
            ldg16(P.bias + n0 + cq, b);
#pragma unroll
            for (int i = 0; i < 16; i += 2) {  // two values per packed FP32 instruction
              float2 h, e;
              celu01_pair(__fadd2_rn(make_float2(v[16 * q + i], v[16 * q + i + 1]), make_float2(b[i], b[i + 1])), h,
                          e);
              v[16 * q + i] = h.x;
              v[16 * q + i + 1] = h.y;
            }
          } else {  // past the problem's columns: zeros
#pragma unroll
            for (int i = 0; i < 16; ++i) v[16 * q + i] = 0.f;
          }
        }
        uint32_t o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          o[i] = Pack<T>::two(v[2 * i], v[2 * i + 1]);
          lo[16 * h32 + i] = Pack<T>::two(v[2 * i] - Pack<T>::lo(o[i]), v[2 * i + 1] - Pack<T>::hi(o[i]));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          *reinterpret_cast<uint4*>(stg + sw128_offset(r, h32 * 32 + 8 * k)) =
              make_uint4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      half_sync();
      if (leader) {
        tma_store_2d(dmap, stg, P.d_col0 + n0 + bx * 64, row);
        bulk_commit();
        in_flight = true;
      }
      if (two) {
        if (leader) bulk_wait_read();  // the hi box has been read
        half_sync();
#pragma unroll
        for (int k = 0; k < 8; ++k)
          *reinterpret_cast<uint4*>(stg + sw128_offset(r, 8 * k)) =
              make_uint4(lo[4 * k], lo[4 * k + 1], lo[4 * k + 2], lo[4 * k + 3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        half_sync();
        if (leader) {
          tma_store_2d(dmap, stg, P.d_col0 + n0 + bx * 64 + P.d_lo, row);
          bulk_commit();
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ TcMaps maps, const GemmProblem* __restrict__ probs,
              const GemmTile* __restrict__ tiles, const int* __restrict__ cta_off, int b_box_rows,
              unsigned* __restrict__ status, const int* __restrict__ abort_req) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // rounded up to 1024 bytes by pointer arithmetic, so that accesses through
  // it stay shared-memory accesses
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* stg_base = smem + kStages * kStageBytes;  // [2] output staging boxes
  uint64_t* full = reinterpret_cast<uint64_t*>(stg_base + 2 * kStgBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;  // [2] accumulator ready
  uint64_t* tempty = tfull + 2;       // [2] accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t stage_tx = kABytes + (uint32_t)b_box_rows * kBK * 2;
  const int tile_begin = cta_off[blockIdx.x], tile_end = cta_off[blockIdx.x + 1];  // this CTA's tiles

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEpiWarps);  // one arrival per epilogue warp
    }
    *abort_flag = *abort_req;  // nonzero only in tests of the abort path
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * kBNMax)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // prologue done: the next kernel may launch; the inputs (and the outputs'
  // previous readers) belong to the kernels before this one
  pdl_launch_dependents();
  pdl_wait();

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      uint32_t it = 0;
      // an abort requested at the start: nothing is loaded (the other roles'
      // first waits give up on the flag)
      const bool pre = *(volatile int*)abort_flag != 0;
      if (pre) atomicOr(status, kStatTimeout);
      for (int tile = pre ? tile_end : tile_begin; tile < tile_end; ++tile) {
        const GemmTile tl = tiles[tile];
        const GemmProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
        const int nkb = (P.K + kBK - 1) / kBK;
        const int ay = P.a_row0 + tl.m0, by = P.b_row0 + tl.n0;
        bool ok = true;
        // K blocks of the segments (A_hi, B_hi), then (A_lo, B_hi) and (A_hi, B_lo)
        // when the operands are split
        const int nseg = P.split ? 3 : 1;
        for (int kt = 0; kt < nseg * nkb; ++kt, ++it) {
          const int seg = kt / nkb, kb = kt - seg * nkb;
          const int s = it % kStages;
          const uint32_t use = it / kStages;
          if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          unsigned char* sa = smem + s * kStageBytes;
          mbar_expect_tx(&full[s], stage_tx);
          tma_load_2d(sa, &maps.a, P.a_col0 + kb * kBK + (seg == 1 ? P.a_lo : 0), ay, &full[s]);
          tma_load_2d(sa + kABytes, &maps.b, P.b_col0 + kb * kBK + (seg == 2 ? P.b_lo : 0), by, &full[s]);
        }
        if (!ok) {
          atomicOr(status, kStatTimeout);
          atomicExch(abort_flag, 1);
          break;
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: the whole warp walks the loop, so that its values stay
    // warp-uniform, and one elected lane issues each instruction ----
    uint32_t it = 0, tcount = 0;
    for (int tile = tile_begin; tile < tile_end; ++tile, ++tcount) {
      const GemmTile tl = tiles[tile];
      const GemmProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
      const int nkb = (P.K + kBK - 1) / kBK;
      const int n_tile = tl.width > 0 ? tl.width : min(b_box_rows, P.N - tl.n0);
      const uint32_t idesc = instr_desc(Pack<T>::fmt, (uint32_t)n_tile);
      const uint32_t acc = tcount & 1, use = tcount >> 1;
      bool ok = use == 0 || mbar_wait_warp(&tempty[acc], (use - 1) & 1, abort_flag);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dtm = tmem + acc * kBNMax;
      const int nkt = (P.split ? 3 : 1) * nkb;
      for (int kt = 0, kb = 0; ok && kt < nkt; ++kt, ++it, kb = kb + 1 == nkb ? 0 : kb + 1) {
        const int s = it % kStages;
        if (!mbar_wait_warp(&full[s], (it / kStages) & 1, abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned char* sa = smem + s * kStageBytes;
        const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sa + kABytes);
        if (kb * kBK + kBK <= P.K) {  // a whole K block: four K = 16 steps, +32 bytes each
          mma_f16_elect4(dtm, da, db, idesc, kt > 0 ? 1u : 0u);
        } else {
          const int ksteps = (P.K - kb * kBK) / 16;
          for (int j = 0; j < ksteps; ++j)
            mma_f16_elect(dtm, da + (uint64_t)(2 * j), db + (uint64_t)(2 * j), idesc,
                          (kt > 0 || j > 0) ? 1u : 0u);
        }
        mma_commit_elect(&empty[s]);
      }
      if (!ok) {
        if (lane == 0) {
          atomicOr(status, kStatTimeout);
          atomicExch(abort_flag, 1);
        }
        break;
      }
      mma_commit_elect(&tfull[acc]);
    }
  } else {
    // ---- epilogue warps 2..9: TMEM lane quarter = warp % 4; half h takes the
    // output boxes h, h + 2, ... of each tile through staging buffer h ----
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int r = quarter * 32 + lane;  // tile row = TMEM lane
    unsigned char* stg = stg_base + half * kStgBytes;
    const bool leader = quarter == 0 && lane == 0;  // issues this half's stores
    bool in_flight = false;                         // leader: a store may still read stg
    auto half_sync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(2 + half) : "memory"); };
    auto epi_sync = [&]() { asm volatile("bar.sync 4, %0;" ::"r"(32 * kEpiWarps) : "memory"); };
    auto epi_any = [&](bool p) -> bool {  // true on every epilogue thread if p on any
      int res;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
          "bar.red.or.pred q, 5, %2, p;\n\tselp.b32 %0, 1, 0, q;\n\t}\n"
          : "=r"(res)
          : "r"(p ? 1 : 0), "r"(32 * kEpiWarps)
          : "memory");
      return res != 0;
    };
    uint32_t tcount = 0;
    for (int tile = tile_begin; tile < tile_end; ++tile, ++tcount) {
      const GemmTile tl = tiles[tile];
      const GemmProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
      const int n_tile = tl.width > 0 ? tl.width : min(b_box_rows, P.N - tl.n0);
      const uint32_t acc = tcount & 1, use = tcount >> 1;
      // the warp (tcgen05.ld is .sync.aligned) and then all epilogue warps
      // agree, so that every named barrier below is reached by all of them
      const bool got = __all_sync(0xffffffffu, mbar_wait(&tfull[acc], use & 1, abort_flag));
      if (!got && lane == 0) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
      }
      if (epi_any(!got)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tbase = tmem + acc * kBNMax + ((uint32_t)(quarter * 32) << 16);
      epi_store_tile<T>(P, tl.n0, n_tile, tbase, stg, r, half, leader, in_flight, &maps.d, P.a_row0 + tl.m0);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
    if (leader && in_flight) bulk_wait_all();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * kBNMax)));
  }
}

// The first layer's products on CTA pairs (thread-block clusters of two):
// each tcgen05.mma.cta_group::2 computes a 256-row tile, rows 0-127 in the
// first CTA's tensor memory and 128-255 in the second's, with B's rows split
// between the two CTAs' shared memory.  Per SM, a 128 x N x 16 step then
// moves 8 KB of operands through shared memory instead of 12 KB (A 4 KB, B
// 4 KB), which lifts the single-CTA kernel's shared-memory cap (192 bytes
// per tensor cycle against 128) to the tensor rate.  Roles as in k_gemm_tc,
// in both CTAs, except:
//   * producers: each CTA loads its own A rows and B half; the first CTA's
//     full[s] counts both CTAs' bytes (the second CTA's loads complete on it
//     through the pair form of the TMA load);
//   * MMA: issued by the first CTA alone; each commit arrives on the barrier
//     at the same offset in both CTAs (stage release, accumulator ready);
//   * epilogue: each CTA drains its own 128 rows and arrives on the first
//     CTA's accumulator-drained barrier (16 arrivals); rows of the second CTA
//     that lie past the element's atoms are not stored.
// Both CTAs walk the same tile list; every wait is bounded as in k_gemm_tc.
// The CTAs leave together (cluster barrier), after the last remote arrival.
template <typename T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_gemm_tc2(const __grid_constant__ TcMaps maps, const GemmProblem* __restrict__ probs,
               const GemmTile* __restrict__ tiles, const int* __restrict__ pair_off, int b_half_rows,
               unsigned* __restrict__ status, const int* __restrict__ abort_req) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* stg_base = smem + kStages2 * kStageBytes2;  // [2] output staging boxes
  uint64_t* full = reinterpret_cast<uint64_t*>(stg_base + 2 * kStgBytes);
  uint64_t* empty = full + kStages2;
  uint64_t* tfull = empty + kStages2;  // [2] accumulator ready (both CTAs)
  uint64_t* tempty = tfull + 2;        // [2] accumulator drained (first CTA's, both CTAs arrive)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const bool first = rank == 0;
  const uint32_t pair_tx = 2 * (kABytes + (uint32_t)b_half_rows * kBK * 2);  // both CTAs' bytes per stage
  const int pair = blockIdx.x >> 1;
  const int tile_begin = pair_off[pair], tile_end = pair_off[pair + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages2; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 2 * kEpiWarps);  // one arrival per epilogue warp of the pair
    }
    *abort_flag = *abort_req;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {  // a pair allocation: one warp of each CTA
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * kBNMax)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();  // both CTAs' barriers exist before any remote arrival
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  pdl_launch_dependents();
  pdl_wait();

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer (both CTAs) ----
      uint32_t it = 0;
      const bool pre = *(volatile int*)abort_flag != 0;
      if (pre) atomicOr(status, kStatTimeout);
      for (int tile = pre ? tile_end : tile_begin; tile < tile_end; ++tile) {
        const GemmTile tl = tiles[tile];
        const GemmProblem P = probs[tl.problem];
        const int nkb = (P.K + kBK - 1) / kBK;
        const int n_tile = tl.width > 0 ? tl.width : min(2 * b_half_rows, P.N - tl.n0);
        const int ay = P.a_row0 + tl.m0 + (int)rank * kBM, by = P.b_row0 + tl.n0 + (int)rank * (n_tile / 2);
        bool ok = true;
        const int nseg = P.split ? 3 : 1;
        for (int kt = 0; kt < nseg * nkb; ++kt, ++it) {
          const int seg = kt / nkb, kb = kt - seg * nkb;
          const int s = it % kStages2;
          const uint32_t use = it / kStages2;
          if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          unsigned char* sa = smem + s * kStageBytes2;
          if (first) mbar_expect_tx(&full[s], pair_tx);
          const uint32_t fb = mapa_rank(&full[s], 0);
          tma_load_2d_pair(sa, &maps.a, P.a_col0 + kb * kBK + (seg == 1 ? P.a_lo : 0), ay, fb);
          tma_load_2d_pair(sa + kABytes, &maps.b, P.b_col0 + kb * kBK + (seg == 2 ? P.b_lo : 0), by, fb);
        }
        if (!ok) {
          atomicOr(status, kStatTimeout);
          atomicExch(abort_flag, 1);
          break;
        }
      }
    }
  } else if (warp == 1) {
    if (first) {
      // ---- MMA issuer (first CTA; whole warp, one elected lane issues) ----
      uint32_t it = 0, tcount = 0;
      for (int tile = tile_begin; tile < tile_end; ++tile, ++tcount) {
        const GemmTile tl = tiles[tile];
        const GemmProblem P = probs[tl.problem];
        const int nkb = (P.K + kBK - 1) / kBK;
        const int n_tile = tl.width > 0 ? tl.width : min(2 * b_half_rows, P.N - tl.n0);
        const uint32_t idesc = instr_desc_m256(Pack<T>::fmt, (uint32_t)n_tile);
        const uint32_t acc = tcount & 1, use = tcount >> 1;
        bool ok = use == 0 || mbar_wait_warp(&tempty[acc], (use - 1) & 1, abort_flag);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dtm = tmem + acc * kBNMax;
        const int nkt = (P.split ? 3 : 1) * nkb;
        for (int kt = 0, kb = 0; ok && kt < nkt; ++kt, ++it, kb = kb + 1 == nkb ? 0 : kb + 1) {
          const int s = it % kStages2;
          if (!mbar_wait_warp(&full[s], (it / kStages2) & 1, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned char* sa = smem + s * kStageBytes2;
          const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sa + kABytes);
          if (kb * kBK + kBK <= P.K) {
            mma_f16_pair_elect4(dtm, da, db, idesc, kt > 0 ? 1u : 0u);
          } else {
            const int ksteps = (P.K - kb * kBK) / 16;
            for (int j = 0; j < ksteps; ++j)
              mma_f16_pair_elect(dtm, da + (uint64_t)(2 * j), db + (uint64_t)(2 * j), idesc,
                                 (kt > 0 || j > 0) ? 1u : 0u);
          }
          mma_commit_pair_elect(&empty[s]);
        }
        if (!ok) {
          if (lane == 0) {
            atomicOr(status, kStatTimeout);
            atomicExch(abort_flag, 1);
          }
          break;
        }
        mma_commit_pair_elect(&tfull[acc]);
      }
    }
  } else {
    // ---- epilogue warps 2..9 (both CTAs), as in k_gemm_tc on this CTA's rows ----
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int r = quarter * 32 + lane;
    unsigned char* stg = stg_base + half * kStgBytes;
    const bool leader = quarter == 0 && lane == 0;
    bool in_flight = false;
    auto epi_any = [&](bool p) -> bool {
      int res;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
          "bar.red.or.pred q, 5, %2, p;\n\tselp.b32 %0, 1, 0, q;\n\t}\n"
          : "=r"(res)
          : "r"(p ? 1 : 0), "r"(32 * kEpiWarps)
          : "memory");
      return res != 0;
    };
    uint32_t tcount = 0;
    for (int tile = tile_begin; tile < tile_end; ++tile, ++tcount) {
      const GemmTile tl = tiles[tile];
      const GemmProblem P = probs[tl.problem];
      const int n_tile = tl.width > 0 ? tl.width : min(2 * b_half_rows, P.N - tl.n0);
      const uint32_t acc = tcount & 1, use = tcount >> 1;
      const bool got = __all_sync(0xffffffffu, mbar_wait(&tfull[acc], use & 1, abort_flag));
      if (!got && lane == 0) {
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
      }
      if (epi_any(!got)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tbase = tmem + acc * kBNMax + ((uint32_t)(quarter * 32) << 16);
      const int m_cta = tl.m0 + (int)rank * kBM;  // this CTA's first row in the element block
      if (m_cta < P.M)  // uniform over the CTA: rows past the element's atoms are not stored
        epi_store_tile<T>(P, tl.n0, n_tile, tbase, stg, r, half, leader, in_flight, &maps.d, P.a_row0 + m_cta);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(mapa_rank(&tempty[acc], 0));
    }
    if (leader && in_flight) bulk_wait_all();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // no arrival or product of the pair is still to come
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * kBNMax)));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

size_t tc_maps_bytes() { return sizeof(TcMaps); }

// 2D tensor map over a row-major [rows][cols] array of 16-bit elements with a
// 64-column x box_rows box and 128-byte swizzle.  Returns false on failure.
bool tc_make_map(void* out_map, const void* base, Prec p, uint64_t rows, uint64_t cols,
                 uint64_t row_stride_elems, uint32_t box_rows, uint32_t box_cols, bool swizzle64) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  CUtensorMap* m = static_cast<CUtensorMap*>(out_map);
  std::memset(m, 0, sizeof(*m));
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {row_stride_elems * (p == Prec::F32 ? 4 : 2)};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = p == Prec::F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : p == Prec::BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const CUresult r = fn(m, dt,
                        2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t tc_set_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<__nv_bfloat16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gemm_tc<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gemm_tc2<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kSmemBytes2);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gemm_tc2<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSmemBytes2);
}

// maps: HOST pointer to the layer's {A, B, D} maps (copied into the launch's
// parameters); b_box_rows: rows of the B map's box; CTA c runs the tiles
// cta_off[c] .. cta_off[c + 1] of the (device) tile list.
void launch_gemm_tc(const GemmProblem* probs, const GemmTile* tiles, const int* cta_off, int n_ctas,
                    Prec p, int b_box_rows, const void* maps, unsigned* status, const int* abort_req,
                    cudaStream_t s) {
  if (n_ctas <= 0) return;
  TcMaps m;
  std::memcpy(&m, maps, sizeof(m));
  if (p == Prec::BF16)
    launch_pdl(k_gemm_tc<__nv_bfloat16>, n_ctas, kThreads, kSmemBytes, s, m, probs, tiles, cta_off,
               b_box_rows, status, abort_req);
  else
    launch_pdl(k_gemm_tc<__half>, n_ctas, kThreads, kSmemBytes, s, m, probs, tiles, cta_off,
               b_box_rows, status, abort_req);
}

// SM pairs that can hold a CTA pair of k_gemm_tc2 at the same time (clusters
// are placed within a GPC), or 0 if the query fails.
int tc2_max_pairs(int sms) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * (sms / 2)));
  cfg.blockDim = dim3((unsigned)kThreads);
  cfg.dynamicSmemBytes = kSmemBytes2;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_gemm_tc2<__nv_bfloat16>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// The first layer on CTA pairs: pair q (CTAs 2q, 2q + 1) runs the tiles
// pair_off[q] .. pair_off[q + 1], 256 rows each; b_half_rows: rows of the B
// map's box (half a tile's columns).
void launch_gemm_tc2(const GemmProblem* probs, const GemmTile* tiles, const int* pair_off, int n_pairs,
                     Prec p, int b_half_rows, const void* maps, unsigned* status, const int* abort_req,
                     cudaStream_t s) {
  if (n_pairs <= 0) return;
  TcMaps m;
  std::memcpy(&m, maps, sizeof(m));
  if (p == Prec::BF16)
    launch_pdl(k_gemm_tc2<__nv_bfloat16>, 2 * n_pairs, kThreads, kSmemBytes2, s, m, probs, tiles, pair_off,
               b_half_rows, status, abort_req);
  else
    launch_pdl(k_gemm_tc2<__half>, 2 * n_pairs, kThreads, kSmemBytes2, s, m, probs, tiles, pair_off,
               b_half_rows, status, abort_req);
}

}  // namespace nnp
