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
//   * warps 2-5: epilogue, tcgen05.ld of the rows they own (warp w reads TMEM
//     lanes 32 (w % 4) ...), bias / CELU / CELU' / the output layer fused,
//     stores to global memory; then hand the accumulator back.
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
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;

struct TcMaps {
  CUtensorMap a;
  CUtensorMap b;
};

// Epilogue of one 16-column chunk of one row.
template <typename T>
__device__ __forceinline__ void epilogue_chunk(const GemmProblem& P, int row, int n,
                                               const float (&v)[16], float& head_acc) {
  switch (P.epi) {
    case (int)Epi::BiasCelu: {
      float b[16];
      ldg16(P.bias + n, b);
      uint32_t o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        o[i] = Pack<T>::two(celu01_fast(v[2 * i] + b[2 * i]), celu01_fast(v[2 * i + 1] + b[2 * i + 1]));
      uint4* d = reinterpret_cast<uint4*>(static_cast<T*>(P.D) + (size_t)row * P.ldd + n);
      d[0] = make_uint4(o[0], o[1], o[2], o[3]);
      d[1] = make_uint4(o[4], o[5], o[6], o[7]);
      break;
    }
    case (int)Epi::Head: {
      uint32_t o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float dv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = n + 2 * i + h;
          const float z = v[2 * i + h] + P.bias[c];
          const float ex = celu01_exp(z);  // celu'(z): 1 above zero
          const float w = P.w4[c];
          head_acc = fmaf(w, fmaxf(z, fmaf(0.1f, ex, -0.1f)), head_acc);
          dv[h] = w * ex * P.inv_m;
        }
        o[i] = Pack<T>::two(dv[0], dv[1]);
      }
      uint4* d = reinterpret_cast<uint4*>(static_cast<T*>(P.D) + (size_t)row * P.ldd + n);
      d[0] = make_uint4(o[0], o[1], o[2], o[3]);
      d[1] = make_uint4(o[4], o[5], o[6], o[7]);
      break;
    }
    case (int)Epi::Bias: {
      float4* d = reinterpret_cast<float4*>(static_cast<float*>(P.D) + (size_t)row * P.ldd + n);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        d[i] = make_float4(v[4 * i] + P.bias[n + 4 * i], v[4 * i + 1] + P.bias[n + 4 * i + 1],
                           v[4 * i + 2] + P.bias[n + 4 * i + 2], v[4 * i + 3] + P.bias[n + 4 * i + 3]);
      break;
    }
    case (int)Epi::DCelu: {
      uint4* d = reinterpret_cast<uint4*>(static_cast<T*>(P.D) + (size_t)row * P.ldd + n);
      const uint4 h0 = d[0], h1 = d[1];
      const uint32_t hin[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
      uint32_t o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float ha = Pack<T>::lo(hin[i]), hb = Pack<T>::hi(hin[i]);
        // celu' from celu (alpha 0.1): 1 + h / alpha below zero, where it is <= 1
        const float ga = fminf(fmaf(10.f, ha, 1.f), 1.f);
        const float gb = fminf(fmaf(10.f, hb, 1.f), 1.f);
        o[i] = Pack<T>::two(v[2 * i] * ga, v[2 * i + 1] * gb);
      }
      d[0] = make_uint4(o[0], o[1], o[2], o[3]);
      d[1] = make_uint4(o[4], o[5], o[6], o[7]);
      break;
    }
    default: {
      float4* d = reinterpret_cast<float4*>(static_cast<float*>(P.D) + (size_t)row * P.ldd + n);
#pragma unroll
      for (int i = 0; i < 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      break;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ TcMaps maps, const GemmProblem* __restrict__ probs,
              const GemmTile* __restrict__ tiles, int n_tiles, int b_box_rows,
              unsigned* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;  // [2] accumulator ready
  uint64_t* tempty = tfull + 2;       // [2] accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t stage_tx = kABytes + (uint32_t)b_box_rows * kBK * 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEpiWarps);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
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

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      uint32_t it = 0;
      for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const GemmTile tl = tiles[tile];
        const GemmProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
        const int nkb = (P.K + kBK - 1) / kBK;
        const int ay = P.a_row0 + tl.m0, by = P.b_row0 + tl.n0;
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages;
          const uint32_t use = it / kStages;
          if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          unsigned char* sa = smem + s * kStageBytes;
          mbar_expect_tx(&full[s], stage_tx);
          tma_load_2d(sa, &maps.a, P.a_col0 + kb * kBK, ay, &full[s]);
          tma_load_2d(sa + kABytes, &maps.b, P.b_col0 + kb * kBK, by, &full[s]);
        }
        if (!ok) {
          atomicOr(status, kStatTimeout);
          atomicExch(abort_flag, 1);
          break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      uint32_t it = 0, tcount = 0;
      for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++tcount) {
        const GemmTile tl = tiles[tile];
        const GemmProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
        const int nkb = (P.K + kBK - 1) / kBK;
        const int n_tile = min(b_box_rows, P.N - tl.n0);  // tile width = weight-box rows
        const uint32_t idesc = instr_desc(Pack<T>::fmt, (uint32_t)n_tile);
        const uint32_t acc = tcount & 1, use = tcount >> 1;
        bool ok = use == 0 || mbar_wait(&tempty[acc], (use - 1) & 1, abort_flag);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dtm = tmem + acc * kBNMax;
        for (int kb = 0; ok && kb < nkb; ++kb, ++it) {
          const int s = it % kStages;
          if (!mbar_wait(&full[s], (it / kStages) & 1, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned char* sa = smem + s * kStageBytes;
          const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sa + kABytes);
          const int ksteps = min(kBK, P.K - kb * kBK) / 16;
          for (int j = 0; j < ksteps; ++j)  // +32 bytes per K step inside the swizzle atom
            mma_f16(dtm, da + (uint64_t)(2 * j), db + (uint64_t)(2 * j), idesc,
                    (kb > 0 || j > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) {
          atomicOr(status, kStatTimeout);
          atomicExch(abort_flag, 1);
          break;
        }
        mma_commit(&tfull[acc]);
      }
    }
  } else {
    // ---- epilogue warps 2..9: TMEM lane quarter = warp % 4, column half ----
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    uint32_t tcount = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++tcount) {
      const GemmTile tl = tiles[tile];
      const GemmProblem P = probs[tl.problem];  // by value: asm memory clobbers force reloads of references
      const int n_tile = min(b_box_rows, P.N - tl.n0);  // tile width = weight-box rows
      const uint32_t acc = tcount & 1, use = tcount >> 1;
      const bool got = mbar_wait(&tfull[acc], use & 1, abort_flag);
      if (!__all_sync(0xffffffffu, got)) {  // the warp leaves together (tcgen05.ld is .sync.aligned)
        atomicOr(status, kStatTimeout);
        atomicExch(abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int epi = P.epi;
      const int row = tl.m0 + quarter * 32 + lane;
      const bool row_ok = row < P.M;
      const uint32_t tbase = tmem + acc * kBNMax + ((uint32_t)(quarter * 32) << 16);
      // column range of this warp: the output layer needs whole rows (first half only)
      int c0 = 0, c1 = n_tile;
      if (epi != (int)Epi::Head) {
        c0 = half * (n_tile >> 1);
        c1 = c0 + (n_tile >> 1);
      } else if (half) {
        c1 = 0;
      }
      if (epi == (int)Epi::DCelu) {
        // prefetch the stored activations of every chunk before the first use
        uint4 hv[2 * (kBNMax / 32)];
#pragma unroll
        for (int i = 0; i < kBNMax / 32; ++i) {
          const int c = c0 + 16 * i;
          if (row_ok && c < c1) {
            const uint4* d = reinterpret_cast<const uint4*>(static_cast<const T*>(P.D) +
                                                           (size_t)row * P.ldd + tl.n0 + c);
            hv[2 * i] = d[0];
            hv[2 * i + 1] = d[1];
          }
        }
#pragma unroll
        for (int i = 0; i < kBNMax / 32; ++i) {
          const int c = c0 + 16 * i;
          if (c >= c1) break;
          float v[16];
          tmem_ld16(tbase + (uint32_t)c, v);
          if (!row_ok) continue;
          const uint32_t hin[8] = {hv[2 * i].x, hv[2 * i].y, hv[2 * i].z, hv[2 * i].w,
                                   hv[2 * i + 1].x, hv[2 * i + 1].y, hv[2 * i + 1].z,
                                   hv[2 * i + 1].w};
          uint32_t o[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float ha = Pack<T>::lo(hin[k]), hb = Pack<T>::hi(hin[k]);
            const float ga = fminf(fmaf(10.f, ha, 1.f), 1.f);  // celu' from celu, alpha 0.1
            const float gb = fminf(fmaf(10.f, hb, 1.f), 1.f);
            o[k] = Pack<T>::two(v[2 * k] * ga, v[2 * k + 1] * gb);
          }
          uint4* d = reinterpret_cast<uint4*>(static_cast<T*>(P.D) + (size_t)row * P.ldd + tl.n0 + c);
          d[0] = make_uint4(o[0], o[1], o[2], o[3]);
          d[1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
      } else {
        float head_acc = 0.f;
        for (int c = c0; c < c1; c += 16) {
          float v[16];
          tmem_ld16(tbase + (uint32_t)c, v);  // all lanes take part (sync.aligned)
          if (row_ok) epilogue_chunk<T>(P, row, tl.n0 + c, v, head_acc);
        }
        if (epi == (int)Epi::Head && half == 0 && row_ok) P.y[(size_t)row * P.ldy] = head_acc + P.b4;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
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
  const cuuint64_t strides[1] = {row_stride_elems * 2};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, p == Prec::BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
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
  return cudaFuncSetAttribute(k_gemm_tc<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSmemBytes);
}

// maps: HOST pointer to the layer's {A map, B map} pair (copied into the
// launch's parameters); b_box_rows: rows of the B map's box.
void launch_gemm_tc(const GemmProblem* probs, const GemmTile* tiles, int n_tiles, Prec p,
                    int b_box_rows, const void* maps, unsigned* status, cudaStream_t s) {
  if (n_tiles <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  TcMaps m;
  std::memcpy(&m, maps, sizeof(m));
  const int grid = n_tiles < sms ? n_tiles : sms;
  if (p == Prec::BF16)
    k_gemm_tc<__nv_bfloat16><<<grid, kThreads, kSmemBytes, s>>>(m, probs, tiles, n_tiles, b_box_rows,
                                                                status);
  else
    k_gemm_tc<__half><<<grid, kThreads, kSmemBytes, s>>>(m, probs, tiles, n_tiles, b_box_rows, status);
}

}  // namespace nnp
