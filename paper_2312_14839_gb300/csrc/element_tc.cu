// FP32 element Hessian with its contraction on the fifth-generation tensor cores (App. B.2).
//
// The element Hessian of one patch is K[(I, c), (J, d)] = sum_g sum_{k, l} phi_gk^I M_g[(k, c), (l, d)]
// phi_gl^J (+ the mass term sum_g m_g phi_g^I phi_g^J delta_cd), with the 16 scalar shape
// functions I, J of the patch, the derivative kinds k, l in {,1 ,2 ,11 ,22 ,12}, the components
// c, d and the 15x15 Gauss-point matrices M_g built exactly as in the FFMA kernel. For each of the
// six component pairs c <= d it is a product of two matrices over the 96 indices (g, k) (16 Gauss
// points x the five derivative kinds plus the value kind that carries the mass):
//   K^{cd}[I][J] = sum_{(g,k)} Psi[(g,k)][I] T^{cd}[(g,k)][J],
//   Psi[(g,k)][I] = phi_gk^I                      (the same for every patch of the shell),
//   T^{cd}[(g,k)][J] = sum_l M_g[(k,c),(l,d)] phi_gl^J   (value kind: m_g phi_g^J delta_cd).
// The threads form T (one row (c, d, J) per thread, 5 multiply-adds per entry) and store it in
// tensor memory; tcgen05.mma (kind::tf32, A = T from tensor memory, B = Psi from shared memory,
// FP32 accumulator in tensor memory) contracts it with Psi. FP32 accuracy from TF32 inputs: both
// operands are split into a TF32 head and a TF32 tail (x = hi + lo), and three products are
// accumulated, T_hi Psi_hi + T_lo Psi_hi + T_hi Psi_lo. Psi_hi is Psi rounded to TF32; T_hi is T
// with its low 13 mantissa bits cleared, and T_lo = T - T_hi (exact), whose low bits the tensor
// core ignores (it reads the top 19 bits of each 32-bit input). The dropped T_lo Psi_lo and the
// truncation of T_lo are below 2^-19 of the product.
//
// CTA: 4 warps, one patch each. Tensor memory (128 columns, so three CTAs share an SM):
//   D (accumulator), tile t = 0..2: columns 16 t .. 16 t + 15,
//   A operand of the current K step, tile t: T_hi at 48 + 16 t (8 columns), T_lo at 56 + 16 t.
// Tile t holds in lane quarter w (warp w's patch) the rows (cd, J) with cd = 2 t + lane / 16 and
// J = lane % 16: 3 tiles of 128 rows for the 96 rows of each of the 4 patches. The K dimension is
// ordered (Gauss-point group gq of 4 points, kind k, point gi): K index 24 gq + 4 k + gi, and one
// step of K = 8 covers two kinds of one group. Per step every warp computes its rows' 8 values
// while the previous step's MMAs run, waits on the mbarrier those MMAs commit to, writes the values
// (head and tail) into the A columns, the CTA synchronises, and one thread issues the step's 9
// MMAs (3 tiles x 3 products) and commits them. After the last step the warps read their accumulator rows back (tcgen05.ld), stage the
// symmetric 48x48 matrix in shared memory and write or scatter it as the FFMA kernel does.
//
// Psi in shared memory: K-major, 128-byte swizzle (the canonical layout of the tcgen05 shared-memory
// descriptor): 3 chunks of 32 K values x 16 rows (128-byte rows, 8-row atoms of 1024 bytes, the
// 16-byte pieces of row n XOR-permuted by n mod 8), head then tail, 12 KB.
//
// Every mbarrier wait is bounded (Shell::wait_polls polls): on expiry the CTA raises
// ERRBIT_TIMEOUT, waits (with the full drain budget) for the MMAs it committed, frees its tensor
// memory and leaves the kernel.
#include "element_impl.cuh"
#include "tc_gemm.cuh"

namespace bhem {
namespace etc {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kTmemCols = 128;
constexpr int kCtasPerSm = 3;
constexpr int kColD = 0;
constexpr int kColA = 48;
constexpr int kPsiBytes = 3 * 2048;   // one of Psi_hi, Psi_lo

// Per-warp shared memory: M_g in the component-pair block layout; the staged 48x48 Hessian and
// the FP64 by-product scratch overlay it.
struct WarpSmemTc {
  float u[48];
  float qb[48];
  float Mb[16][kMbG];
  float G[16][15];
  float ms[16];
  float en[16];
};
static_assert(sizeof(WarpSmemTc::Mb) >= sizeof(float) * 48 * kKStride, "staging area");
static_assert(sizeof(WarpSmemTc::Mb) >= 2 * 432 * sizeof(double), "FP64 scratch");
static_assert(sizeof(WarpSmemTc) % 16 == 0 && offsetof(WarpSmemTc, Mb) % 16 == 0, "16-byte block loads");

constexpr size_t kSmemBytes =
    1024 + 2 * kPsiBytes + sizeof(float) * ((kPhiTable + 3) & ~3) + sizeof(WarpSmemTc) * kWarps;
// the resident CTAs of an SM: their tensor memory (512 columns per SM), their shared memory
// (228 KB per SM, 1 KB of it reserved per CTA, about 1 KB of static arrays each) and their
// registers (64K per SM at the 168 the launch bounds allow)
static_assert(kCtasPerSm * kTmemCols <= 512, "tensor memory of the resident CTAs");
static_assert(kCtasPerSm * (kSmemBytes + 2048) <= 228 * 1024, "shared memory of the resident CTAs");
static_assert(kCtasPerSm * kThreads * 168 <= 65536, "registers of the resident CTAs");

// Instruction descriptor of kind::tf32: TF32 A and B, FP32 D, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// D (tensor memory) += A (tensor memory) B (shared-memory descriptor); acc = false overwrites D.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"((uint32_t)acc)
      : "memory");
}

// 8 consecutive 32-bit columns of this thread's lane (warp-collective; address of the warp's
// lane quarter).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// component pair of index cd (c <= d)
__device__ __forceinline__ int cd_c(int cd) { return cd < 3 ? 0 : (cd < 5 ? 1 : 2); }
__device__ __forceinline__ int cd_d(int cd) { return cd < 3 ? cd : (cd < 5 ? cd - 2 : 2); }

__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_element_tc(ElemArgs A, unsigned polls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ double w1_64[kHerm1D], w2_64[kHerm1D];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t raw = tc::smem_addr(smem_raw);
  const uint32_t bbase = (raw + 1023u) & ~1023u;
  unsigned char* bptr = smem_raw + (bbase - raw);
  float* sphi = reinterpret_cast<float*>(bptr + 2 * kPsiBytes);
  WarpSmemTc* Ws = reinterpret_cast<WarpSmemTc*>(sphi + ((kPhiTable + 3) & ~3));

  load_shape_table<float>(sphi, reinterpret_cast<const float*>(A.phi));
  if (A.grad64) {
    build_hermite_1d<double>(w1_64, A.d1, tid, kThreads);
    build_hermite_1d<double>(w2_64, A.d2, tid, kThreads);
  }
  __syncthreads();
  // B operand: Psi[(g, k)][I] at K index 24 gq + 4 k + gi (g = 4 gq + gi; k = 5: the value phi)
  for (int e = tid; e < 16 * 96; e += kThreads) {
    const int n = e / 96, kk = e % 96;
    const int gq = kk / 24, r = kk % 24, k = r >> 2, g = 4 * gq + (r & 3);
    const float v = k < 5 ? sphi[n * kPhiStride + (k + 1) * 16 + g] : sphi[n * kPhiStride + g];
    const float hi = to_tf32(v), lo = to_tf32(v - hi);
    const int off = (kk >> 5) * 2048 + n * 128 + ((((kk & 31) >> 2) ^ (n & 7)) << 4) + (kk & 3) * 4;
    *reinterpret_cast<float*>(bptr + off) = hi;
    *reinterpret_cast<float*>(bptr + kPsiBytes + off) = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(&bar_mma), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (wid == 0) tc::tmem_alloc<kTmemCols>(tc::smem_addr(&tmem_slot));
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t tq = tmem + ((uint32_t)(32 * wid) << 16);   // this warp's lane quarter
  const uint32_t bar = tc::smem_addr(&bar_mma);
  constexpr uint32_t idesc = idesc_tf32(128, 16);

  WarpSmemTc& W = Ws[wid];
  const int cdl = lane >> 4, J = lane & 15;
  const int total = A.plist ? A.plist_n : A.np;
  const int stride = gridDim.x * kWarps;
  uint32_t phase = 0;
  bool bad = false, aborted = false;
  int k2 = 0;
  for (int base = blockIdx.x * kWarps; base < total && !aborted; base += stride, ++k2) {
    const int it = base + wid;
    const bool active = it < total;
    const int p = active ? (A.plist ? A.plist[it] : it) : 0;
    if (A.grad64 && (k2 & 1) == 0) {
      // FP64 energy and gradient at the same q (as in k_element_full): every second patch of a
      // warp, its two half-warps evaluate that patch and the warp's next one
      const int hw = lane >> 4, g = lane & 15;
      double* scratch = reinterpret_cast<double*>(&W.Mb[0][0]) + hw * 432;
      const int itp = it + hw * stride;
      const bool act = itp < total;
      const int pp = act ? (A.plist ? A.plist[itp] : itp) : 0;
      int nd[4] = {0, 0, 0, 0};
      if (act) {
        const int4 pn = A.pnodes[pp];
        nd[0] = pn.x;
        nd[1] = pn.y;
        nd[2] = pn.z;
        nd[3] = pn.w;
      }
      const double ep = eg64_patch(w1_64, w2_64, scratch, scratch + 48,
                                   reinterpret_cast<double(*)[15]>(scratch + 192), pp, act, g, nd, A.q, nullptr,
                                   0.0, A.restgp, (size_t)A.np * 16, A.h, A.grad64, A.err);
      if (act && g == 0) {
        if (!isfinite(ep)) atomicOr(A.err, ERRBIT_NONFINITE);
        A.energy64[pp] = ep;
      }
      __syncwarp();
    }
    if (active) {
      gather_patch<float>(W, p, A, lane);
      __syncwarp();
      gauss_point_matrix<float, true, true>(sphi, W, lane & 15, lane >> 4, A);
      __syncwarp();
      patch_byproducts<float>(sphi, W, p, A, lane);
    }

    // T rows into tensor memory, one K step (8 values per row) at a time, and the MMAs. The
    // values of step s are computed while the MMAs of step s - 1 run; the A columns are rewritten
    // once those MMAs have completed.
#pragma unroll 1
    for (int s = 0; s < 12; ++s) {
      const int gq = s / 3, j = s - 3 * gq;
      float a[3][8];
      if (active) {
#pragma unroll
        for (int gi = 0; gi < 4; ++gi) {
          const int g = 4 * gq + gi;
          float ph[6];
#pragma unroll
          for (int l = 0; l < 5; ++l) ph[l] = sphi[J * kPhiStride + (l + 1) * 16 + g];
          ph[5] = sphi[J * kPhiStride + g];
          const float mg = W.ms[g];
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int cd = 2 * t + cdl;
            const bool diag = cd == 0 || cd == 3 || cd == 5;
            // the two kinds k = 2j, 2j + 1 of this step: rows m[k][0..4] at 12 j and 12 j + 6
            // (three 16-byte loads; in step 2 the second row is not used)
            const float4* mb = reinterpret_cast<const float4*>(&W.Mb[4 * gq + gi][cd * kBlk + 2 * kBlkRow * j]);
            const float4 f0 = mb[0], f1 = mb[1], f2 = mb[2];
            const float r0[5] = {f0.x, f0.y, f0.z, f0.w, f1.x};
            const float r1[5] = {f1.z, f1.w, f2.x, f2.y, f2.z};
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int l = 0; l < 5; ++l) {
              s0 = fmaf(r0[l], ph[l], s0);
              s1 = fmaf(r1[l], ph[l], s1);
            }
            a[t][gi] = s0;
            // step 2 of a group holds kind 4 and the value kind (mass, diagonal pairs only)
            a[t][4 + gi] = j < 2 ? s1 : (diag ? mg * ph[5] : 0.f);
          }
        }
      }
      if (s > 0) {
        if (!tc::mbar_wait_parity(bar, phase, polls)) bad = true;
        phase ^= 1u;
        tc::tc_fence_after();
      }
      if (active) {
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          // head: the value with its low 13 mantissa bits cleared (a TF32 number); tail: the
          // exact remainder, whose own low bits the tensor core ignores
          float hi[8], lo[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            hi[e] = __uint_as_float(__float_as_uint(a[t][e]) & 0xffffe000u);
            lo[e] = a[t][e] - hi[e];
          }
          tmem_st8(tq + (uint32_t)(kColA + 16 * t), hi);
          tmem_st8(tq + (uint32_t)(kColA + 16 * t + 8), lo);
        }
        tmem_st_wait();
      }
      tc::tc_fence_before();
      if (__syncthreads_or(bad)) {
        aborted = true;
        break;
      }
      if (tid == 0) {
        tc::tc_fence_after();
        const int kk0 = 8 * s;
        const uint32_t boff = (uint32_t)((kk0 >> 5) * 2048 + (kk0 & 31) * 4);
        const uint64_t bh = tc::smem_desc_sw128(bbase + boff);
        const uint64_t bl = tc::smem_desc_sw128(bbase + kPsiBytes + boff);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const uint32_t d = tmem + (uint32_t)(kColD + 16 * t);
          const uint32_t ah = tmem + (uint32_t)(kColA + 16 * t), al = ah + 8;
          mma_tf32_ts(d, ah, bh, idesc, s > 0);
          mma_tf32_ts(d, al, bh, idesc, true);
          mma_tf32_ts(d, ah, bl, idesc, true);
        }
        tc::mma_commit(bar);
      }
    }
    if (aborted) break;
    // the last step's MMAs
    if (!tc::mbar_wait_parity(bar, phase, polls)) bad = true;
    phase ^= 1u;
    tc::tc_fence_after();
    if (__syncthreads_or(bad)) {
      aborted = true;
      break;
    }

    // accumulator rows back: K^{cd}[I][J] for the lane's (cd, J) of each tile
    uint32_t r[3][16];
#pragma unroll
    for (int t = 0; t < 3; ++t) tc::tmem_ld16_async(tq + (uint32_t)(kColD + 16 * t), r[t]);
    tc::tmem_ld_wait();
    if (active) {
      float* K = &W.Mb[0][0];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        // entry (I, c), (J, d) and its mirror; a diagonal pair (c = d) takes the entries I <= J of
        // column J only (one path for both half-warps, whose pairs differ in kind)
        const int cd = 2 * t + cdl, c = cd_c(cd), d = cd_d(cd);
        const bool off = c < d;
#pragma unroll
        for (int I = 0; I < 16; ++I) {
          if (off || I <= J) {
            const float v = __uint_as_float(r[t][I]);
            K[(I * 3 + c) * kKStride + J * 3 + d] = v;
            K[(J * 3 + d) * kKStride + I * 3 + c] = v;
          }
        }
      }
      __syncwarp();
      store_staged_hessian32(K, p, A, lane);
    }
  }
  if (aborted) {
    if (tid == 0) {
      atomicOr(A.err, ERRBIT_TIMEOUT);
      // the MMAs of the step whose wait expired are still pending: wait for their commit
      tc::mbar_wait_parity(bar, phase ^ 1u, tc::kDrainPolls);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (wid == 0) tc::tmem_dealloc<kTmemCols>(tmem);
}

}  // namespace etc

// FP32 element pass with the tensor-core contraction; the arguments as for k_element_full<float>.
shell_status launch_full_tc(Shell& s, const ElemArgs& A, int work) {
  static bool attr_done[64] = {false};
  const int dev = s.device < 64 ? s.device : 63;
  if (!attr_done[dev]) {
    BHEM_CUDA(cudaFuncSetAttribute(etc::k_element_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)etc::kSmemBytes));
    attr_done[dev] = true;
  }
  if (work <= 0) return SHELL_OK;
  if (s.num_sms <= 0) BHEM_CUDA(cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, s.device));
  // three CTAs per SM, all resident (168 registers x 384 threads, 3 x 70 KB of shared memory and
  // 3 x 128 of the 512 tensor-memory columns); each loops over patch groups until the work is done
  int blocks = (work + etc::kWarps - 1) / etc::kWarps;
  const int cap = s.num_sms * etc::kCtasPerSm;
  if (blocks > cap) blocks = cap;
  etc::k_element_tc<<<blocks, etc::kThreads, etc::kSmemBytes, s.stream>>>(A, (unsigned)s.wait_polls);
  BHEM_CUDA(cudaGetLastError());
  ++s.launches;
  return SHELL_OK;
}

}  // namespace bhem
