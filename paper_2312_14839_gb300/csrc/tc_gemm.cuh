// BF16 GEMM on the fifth-generation tensor cores: C[m][n] = sum_k A[m][k] B[n][k], FP32
// accumulation in tensor memory (TMEM). Operands are K-contiguous BF16 matrices in global memory,
// moved into shared memory by TMA tensor copies; one thread issues tcgen05.mma (kind::f16, BF16
// inputs, FP32 accumulator), and the warps of the CTA read the accumulator back with tcgen05.ld
// for the epilogue.
//
// Shared-memory operand layout (128-byte swizzle, K-major canonical form): a K chunk of 64 BF16
// columns is one 128-byte row per matrix row, 8-row atoms of 1024 bytes, the 16-byte pieces of
// row r XOR-permuted by r mod 8. One TMA tensor copy (box 64 columns x rows, SWIZZLE_128B) writes
// a whole operand tile of a stage in this layout; an MMA of K = 16 starts 32 bytes further along
// the row than the previous one.
//
// Pipeline (per CTA): thread 0 issues the TMA copies of up to S K chunks ahead (one mbarrier per
// stage counts the bytes), thread 32 waits for each stage, issues its four MMAs and commits them
// to the stage's "empty" mbarrier, which releases the stage to the producer. A final commit
// signals the epilogue, which all 8 warps share. With 128-column tiles two CTAs fit an SM, so one
// CTA's epilogue (latency-bound: TMEM loads, staging stores, proxy fences, TMA store issue)
// overlaps the other's loads and MMAs. Every wait is bounded: on expiry the CTA raises an error
// bit, waits (bounded) for the copies it issued, skips the epilogue, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdint>

namespace bhem {
namespace tc {

constexpr int kBM = 128;          // rows per CTA tile (TMEM lanes)
constexpr int kThreads = 256;     // 8 warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, column part w / 4
constexpr int kBK = 64;           // K columns per pipeline stage (four MMAs of K = 16), 128 bytes
// Budget of the waits that drain a CTA's own copies after another wait expired: those copies are
// bound to land, so they get the full budget whatever the caller's.
constexpr unsigned kDrainPolls = 1u << 20;

// ---------------------------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// Waits for the completion of the phase with the given parity; false after `polls` failed polls.
__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity, unsigned polls) {
  for (unsigned i = 0; i < polls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle (K-major): rows of 128 bytes, 8-row atoms of
// 1024 bytes (stride byte offset), layout type 2 in bits 61..63; the leading byte offset is unused.
// The start address may step along K inside an atom (32 bytes per K = 16 of BF16).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

template <int COLS>
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "n"(COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

template <int COLS>
__device__ __forceinline__ void tmem_dealloc(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(COLS) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane (warp w reads lanes
// 32 (w % 4) .. + 31), without waiting; all lanes of the warp must execute it.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  tmem_ld16_async(taddr, r);
  tmem_ld_wait();
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// TMA tensor stores from shared memory (bulk groups): plain, and element-wise atomic FP32 add
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// all but the newest N groups have finished reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// every group has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------------------
struct TcShape {
  int M, N;               // output rows and columns
  int kchunks;            // ceil(K / kBK)
  int kchunks_per_split;  // K chunks of one blockIdx.z (the host makes every split non-empty)
  unsigned polls;         // bound of every mbarrier wait
  int* err;               // error word; err_bit is raised when a wait expires
  int err_bit;
  int out_mask;           // TcOutChannel bits: which outputs the epilogue writes
  const float* colvec;    // optional per-column vector [N] handed to the epilogue (e.g. a bias)
};

// Outputs of the epilogue, written by TMA tensor stores from per-warp shared-memory tiles of
// 32 rows x 16 columns: FP32 [M][N] (stored, or added atomically for split K), BF16 [M][N], and
// BF16 transposed [N][M]. Maps from encode_out_map (boxes 16 x 32, and 32 x 16 transposed).
struct TcOut {
  CUtensorMap f32, b16, b16t;
};
enum TcOutChannel : int { kOutF32 = 1, kOutF32Add = 2, kOutB16 = 4, kOutB16T = 8 };

template <int BN>
struct TcCfg {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "N tile of an M = 128 MMA");
  static constexpr int kStages = BN >= 128 ? 3 : 4;
  static constexpr int kBytesA = kBM * kBK * 2;
  static constexpr int kBytesB = BN * kBK * 2;
  static constexpr int kStage = kBytesA + kBytesB;
  static constexpr int kTmemCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  static_assert(kStage % 1024 == 0, "every operand tile starts on a 1024-byte swizzle atom");
  // epilogue: the four warps of a TMEM lane quarter split the columns into kParts parts of whole
  // 16-column groups; each epilogue warp stages two 4 KB slots in the freed operand stages
  static constexpr int kMaxParts = kThreads / 128;
  static constexpr int kParts = BN / 16 < kMaxParts ? BN / 16 : kMaxParts;
  static constexpr int kPartCols = BN / kParts;
  static_assert(kPartCols % 16 == 0, "column parts of whole 16-column TMEM loads");
  static constexpr int kStageWarp = 2 * 4096;
  static constexpr size_t kPipeBytes = (size_t)kStages * kStage;
  static constexpr size_t kEpiBytes = (size_t)kParts * 4 * kStageWarp;
  static constexpr size_t kSmem = (kPipeBytes > kEpiBytes ? kPipeBytes : kEpiBytes) + 1024;   // + base alignment
};

// Epi: a functor with
//   __device__ void operator()(int row, int col0, const float* colvec, const float (&acc)[16],
//                              float (&f32)[16], float (&b16)[16]) const
// that turns accumulator columns col0 .. col0 + 15 of one row into the values of the FP32 channel
// and of the BF16 channels; colvec points at the per-column vector's entry for col0 (shared
// memory). Rows past M are clipped by the stores: for such a row (row >= M) the functor must not
// read memory indexed by it.
template <int BN, class Epi>
__global__ void __launch_bounds__(kThreads, 2)
k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const __grid_constant__ TcOut out, TcShape sh, Epi epi) {
  using C = TcCfg<BN>;
  constexpr int S = C::kStages;
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[S];
  __shared__ __align__(8) uint64_t bar_empty[S];
  __shared__ __align__(8) uint64_t bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort, s_consumed, s_issued;
  __shared__ float s_colvec[BN];
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_addr(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  for (int c = tid; c < BN; c += kThreads) s_colvec[c] = (sh.colvec && n0 + c < sh.N) ? sh.colvec[n0 + c] : 0.f;
  const int kc0 = blockIdx.z * sh.kchunks_per_split;
  const int nk = min(sh.kchunks, kc0 + sh.kchunks_per_split) - kc0;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_addr(&bar_full[s]), 1);
      mbar_init(smem_addr(&bar_empty[s]), 1);
    }
    mbar_init(smem_addr(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
    s_consumed = 0;
    s_issued = 0;
  }
  if (warp == 0) tmem_alloc<C::kTmemCols>(smem_addr(&tmem_slot));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    // producer: TMA copies of K chunk i into stage i % S once the MMAs of chunk i - S are done
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % S;
      if (i >= S && !mbar_wait_parity(smem_addr(&bar_empty[s]), ((i / S) - 1) & 1, sh.polls)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const uint32_t fb = smem_addr(&bar_full[s]);
      mbar_arrive_expect_tx(fb, C::kStage);
      const uint32_t sa = base + s * C::kStage, sb = sa + C::kBytesA;
      const int k0 = (kc0 + i) * kBK;
      tma_load_2d(sa, &tmA, fb, k0, m0);
      tma_load_2d(sb, &tmB, fb, k0, n0);
    }
    s_issued = i;
  } else if (tid == 32) {
    // MMA issuer: four K = 16 MMAs per chunk into the TMEM accumulator
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % S;
      if (!mbar_wait_parity(smem_addr(&bar_full[s]), (i / S) & 1, sh.polls)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = base + s * C::kStage, sb = sa + C::kBytesA;
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j) {
        const uint64_t da = smem_desc_sw128(sa + 32 * j);
        const uint64_t db = smem_desc_sw128(sb + 32 * j);
        mma_bf16_ss(tmem, da, db, idesc, i > 0 || j > 0);
      }
      mma_commit(smem_addr(&bar_empty[s]));
    }
    s_consumed = i;
    mma_commit(smem_addr(&bar_done));
  }
  // every thread: wait for the last MMA (a CTA with nothing consumed still gets the commit)
  if (!mbar_wait_parity(smem_addr(&bar_done), 0, sh.polls)) *abort_flag = 1;
  __syncthreads();
  const bool aborted = *abort_flag != 0;
  if (aborted) {
    if (tid == 0) {
      atomicOr(sh.err, sh.err_bit);
      // copies issued but not consumed, and the final commit, are still landing in shared
      // memory: wait for them before the CTA exits
      for (int i = s_consumed; i < s_issued; ++i)
        mbar_wait_parity(smem_addr(&bar_full[i % S]), (i / S) & 1, kDrainPolls);
      mbar_wait_parity(smem_addr(&bar_done), 0, kDrainPolls);
    }
  } else if (nk > 0) {
    // epilogue: the four warps of a TMEM lane quarter share its columns (parts of >= 16 columns)
    tc_fence_after();
    constexpr int kParts = C::kParts, kPartCols = C::kPartCols;
    const int quarter = warp & 3, part = warp >> 2;
    const int row = m0 + quarter * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    if (part < kParts) {
      // two 4 KB slots per warp, one per 16-column group of a 32-column step: FP32 tile [32][16]
      // at 0, BF16 [32][16] at 2048, BF16 transposed [16][32] at 3072. A step reads its 32
      // accumulator columns with two loads and one wait, fills both slots once the previous
      // step's stores have read them, and publishes them with one proxy fence and one bulk group.
      const uint32_t stg = base + (uint32_t)(part * 4 + quarter) * C::kStageWarp;
      unsigned char* stg_g = tc_smem_raw + (stg - raw);
      const int mask = sh.out_mask;
      const int y = m0 + quarter * 32;
#pragma unroll 1
      for (int cb = part * kPartCols; cb < (part + 1) * kPartCols; cb += 32) {
        if (n0 + cb >= sh.N) break;
        const int ng = (cb + 16 < (part + 1) * kPartCols && n0 + cb + 16 < sh.N) ? 2 : 1;
        uint32_t r[2][16];
        tmem_ld16_async(lane_addr + (uint32_t)cb, r[0]);
        if (ng == 2) tmem_ld16_async(lane_addr + (uint32_t)(cb + 16), r[1]);
        tmem_ld_wait();
        if (cb > part * kPartCols) {
          if (lane == 0) bulk_wait_read<0>();
          __syncwarp();
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h >= ng) break;
          const int c0 = cb + 16 * h;
          float v[16], f[16], b[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[h][j]);
          epi(row, n0 + c0, s_colvec + c0, v, f, b);
          unsigned char* sp = stg_g + h * 4096;
          if (mask & (kOutF32 | kOutF32Add)) {
            float4* d = reinterpret_cast<float4*>(sp + lane * 64);
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
          }
          if (mask & kOutB16) {
            unsigned w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              w[j] = (unsigned)__bfloat16_as_ushort(__float2bfloat16(b[2 * j])) |
                     ((unsigned)__bfloat16_as_ushort(__float2bfloat16(b[2 * j + 1])) << 16);
            uint4* d = reinterpret_cast<uint4*>(sp + 2048 + lane * 32);
            d[0] = make_uint4(w[0], w[1], w[2], w[3]);
            d[1] = make_uint4(w[4], w[5], w[6], w[7]);
          }
          if (mask & kOutB16T) {
            __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(sp + 3072);
#pragma unroll
            for (int j = 0; j < 16; ++j) d[j * 32 + lane] = __float2bfloat16(b[j]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          for (int h = 0; h < ng; ++h) {
            const uint32_t ss = stg + (uint32_t)h * 4096u;
            const int x = n0 + cb + 16 * h;
            if (mask & kOutF32) tma_store_2d(&out.f32, ss, x, y);
            if (mask & kOutF32Add) tma_reduce_add_2d(&out.f32, ss, x, y);
            if (mask & kOutB16) tma_store_2d(&out.b16, ss + 2048, x, y);
            if (mask & kOutB16T) tma_store_2d(&out.b16t, ss + 3072, y, x);
          }
          bulk_commit();
        }
        __syncwarp();
      }
      if (lane == 0) bulk_wait_all();
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc<C::kTmemCols>(tmem);
}

// ---------------------------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------------------------
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Tensor map of a row-major matrix [rows][cols] (row stride ld elements) with boxes of box_cols x
// box_rows; reads outside [0, cols) x [0, rows) return zeros and stores there are dropped. Returns
// false when the driver entry point is missing, the layout breaks a TMA rule (16-byte aligned
// base, row stride a multiple of 16 bytes) or the driver rejects it.
inline bool encode_map(CUtensorMap* map, CUtensorMapDataType type, int elem_bytes, const void* base, long long rows,
                       long long cols, long long ld, int box_cols, int box_rows, CUtensorMapSwizzle swizzle) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !base || rows < 1 || cols < 1 || ld < cols || ((uintptr_t)base & 15) || ((ld * elem_bytes) & 15) ||
      box_rows < 1 || box_rows > 256 || box_cols < 1 || box_cols > 256)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * elem_bytes)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, type, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// GEMM operand: BF16 [rows][cols], K = cols contiguous, read in 64-column boxes of box_rows rows
// into the 128-byte swizzled layout.
inline bool encode_bf16_map(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld,
                            int box_rows) {
  return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, rows, cols, ld, kBK, box_rows,
                    CU_TENSOR_MAP_SWIZZLE_128B);
}

// Epilogue outputs (TcOut): FP32 or BF16 [rows][cols] in 16-column x 32-row boxes; the transposed
// BF16 channel [cols of the GEMM][rows of the GEMM] in 32 x 16 boxes.
inline bool encode_out_f32(CUtensorMap* map, const float* base, long long rows, long long cols, long long ld) {
  return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, rows, cols, ld, 16, 32, CU_TENSOR_MAP_SWIZZLE_NONE);
}
inline bool encode_out_b16(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld) {
  return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, rows, cols, ld, 16, 32,
                    CU_TENSOR_MAP_SWIZZLE_NONE);
}
inline bool encode_out_b16t(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld) {
  return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, rows, cols, ld, 32, 16,
                    CU_TENSOR_MAP_SWIZZLE_NONE);
}

// Launches C = A B^T for A [M][K] (map box 128 rows) and B [N][K] (map box BN rows), splitting K
// over at most ksplit CTAs per output tile (then the FP32 channel must be kOutF32Add). N must be a
// multiple of 16.
template <int BN, class Epi>
inline cudaError_t launch_gemm_tc(const CUtensorMap& a, const CUtensorMap& b, const TcOut& out, int out_mask,
                                  const float* colvec, int M, int N, int K, int ksplit, const Epi& epi, int* err,
                                  int err_bit, unsigned polls, cudaStream_t st) {
  using C = TcCfg<BN>;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!attr_set[dev & 63]) {
    e = cudaFuncSetAttribute(k_gemm_tc<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev & 63] = true;
  }
  if (M < 1 || N < 1 || K < 1) return cudaSuccess;
  if (N % 16) return cudaErrorInvalidValue;
  const int kchunks = (K + kBK - 1) / kBK;
  if (ksplit < 1) ksplit = 1;
  const int per = (kchunks + ksplit - 1) / ksplit;
  const int splits = (kchunks + per - 1) / per;
  const dim3 grid((N + BN - 1) / BN, (M + kBM - 1) / kBM, splits);
  const TcShape sh{M, N, kchunks, per, polls, err, err_bit, out_mask, colvec};
  k_gemm_tc<BN, Epi><<<grid, kThreads, C::kSmem, st>>>(a, b, out, sh, epi);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace bhem
