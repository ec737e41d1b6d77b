// Fast Poisson preconditioner (Sec. 2.2 / Algorithm 1) on the 5th-generation tensor cores.
//
// The four separable transform products of the preconditioner (stage equations in
// kernels_gemm_simt.cu) run as tcgen05 MMAs with FP16 or BF16 operands and FP32 accumulation.
// This operator is so ill-conditioned that a plain 16-bit operand ruins the preconditioner, and
// even float hi/lo operand splits lose too much in the tensor core's truncating FP32
// accumulation.  The products are therefore made exact:
//
//  * every operand is cut into blocks of KC = 128 consecutive k; a block with largest magnitude
//    below 2^E (and 2^(8-E) times it below 255.5) is stored as four integer slices,
//    v = c0 2^(E-8) + c1 2^(E-16) + c2 2^(E-24) + c3 2^(E-32), |c0| <= 255, |c1..c3| <= 128
//    (exact in FP16 and BF16), plus the exponent E (int8);
//  * for each slice order d = i + j <= 3 (products c_i c'_j; higher orders are below 2^-32 of
//    the block and dropped) a separate TMEM accumulator sums one k-block.  The B slices are
//    stacked along N, so the ten products of a k-step take four MMAs (N = 256, 192, 128, 64).
//    Per k, the products of one order add up to less than 2^16.6, so over 128 k every partial
//    sum is an exact integer below 2^24 and so is the accumulation;
//  * the epilogue warps scale the four exact sums by 2^(E_A + E_B - 16 - 8d) and add them into
//    a compensated (hi, lo) register pair, k-block after k-block, two columns per packed FP32x2
//    operation.
// The operands carry 32 bits relative to each 128-block's largest value and the products add no
// error along K; the stage outputs stay double-float (hi, lo) pairs and are sliced from them
// directly, and the last stage writes z as a double-float pair.  Three slices on
// 64-blocks (24 bits) cost this operator 30-80% more CG iterations than exact transforms; four on
// 128-blocks come within 5-10% of them.  The writer of the next stage's operand computes its
// block exponents with a four-warp maximum and stores the slices transposed (Out[n][m],
// coalesced along m).
//
// Kernel structure (one CTA per SM, persistent over the (slot, tile) work list):
//   warp 0      : TMA producer: 128B-swizzled K-major tiles of the four slices of A and B
//   warp 1      : TMEM allocation; lane 0 issues the MMAs and the tcgen05.commit arrivals
//   warps 2..17 : four per TMEM lane quarter (32 rows), each owning 16 of the tile's 64 columns:
//                 exact k-block sums -> compensated registers -> the stage's epilogue
//                 (eigenvalue weights; masking and per-tile r.z, z.q partials in stage 3).
// Every wait on an mbarrier is bounded; on time-out the CTA raises an error flag, drains its
// outstanding copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "async.cuh"
#include "common.cuh"
#include "kernels.h"

namespace bx {
namespace {

constexpr int BM = 128, BN = 64, BK = 64;  // BK: one 128-byte swizzle atom per pipeline stage
constexpr int KC = 128;                     // k per exponent / exact accumulation block
constexpr int KPC = KC / BK;                // pipeline stages per accumulation block
constexpr int NS = 4;                            // slices per operand
constexpr int kEpiWarps = 16;
constexpr int kColGroups = kEpiWarps / 4;        // epilogue warps per TMEM lane quarter
constexpr int kEpiCols = BN / kColGroups;        // tile columns per epilogue warp
static_assert(kEpiCols % 16 == 0 && kEpiCols <= 32, "epilogue column split");
static_assert(KC % BK == 0 && KC <= BM && BM % KC == 0, "exponent blocks within a tile");
constexpr int kLdCols = kEpiWarps == 16 ? 4 : 8;  // TMEM columns per load (register budget)
constexpr int kThreads = 64 + 32 * kEpiWarps;
// One CTA per SM.  Each of the SM's four schedulers owns a quarter of the register file and
// holds up to ceil(warps / 4) of the CTA's warps.
constexpr int kMaxRegs = (16384 / (32 * ((kThreads / 32 + 3) / 4))) & ~7;
constexpr int kChunks = 2;                       // TMEM ring of k-block accumulator sets
constexpr int kSetCols = NS * BN;                // one accumulator per slice order
constexpr int kTmemCols = 512;                   // power of two >= kChunks * kSetCols
static_assert(kChunks * kSetCols <= kTmemCols, "TMEM columns");
constexpr int STAGES = 2;
constexpr int A_PLANE = BM * BK * 2;
constexpr int B_PLANE = BN * BK * 2;
constexpr int STAGE_BYTES = NS * (A_PLANE + B_PLANE);
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 2048;

struct Ctl {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[kChunks];
  uint64_t tempty[kChunks];
  uint64_t drain;
  uint32_t tmem;
  int abort_flag;
  int last;
  int pad;
  float red[kEpiWarps][4];  // stage 3: per-warp compensated r.z and z.q
  float colmax[kColGroups][4][kEpiCols];  // [column group][lane quarter][column]
};
static_assert(sizeof(Ctl) <= 2048, "control block too large");

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row core groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;          // leading-dimension offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;  // stride between 8-row groups
  d |= static_cast<uint64_t>(1) << 46;          // descriptor version
  d |= static_cast<uint64_t>(2) << 61;          // 128-byte swizzle
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, both operands K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int M, int N) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
[[maybe_unused]] __device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15])
      : "r"(taddr));
}
[[maybe_unused]] __device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&v)[N]) {
  if constexpr (N == 16) tmem_ld16(taddr, v);
  else if constexpr (N == 8) tmem_ld8(taddr, v);
  else tmem_ld4(taddr, v);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// A global load that stays where it is written (volatile asm is not moved across the other
// volatile asm of the k-block loop), so its latency overlaps the loop.
__device__ __forceinline__ float ld_early(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

// 2^e as a float for e in the normal range, 0 below it.
__device__ __forceinline__ float pow2f(int e) {
  return e < -126 ? 0.f : __int_as_float((min(e, 127) + 127) << 23);
}

// Exponent E of a block whose largest magnitude is amax: amax < 2^E (0 for an all-zero block);
// for blocks wider than 64 also amax 2^(8-E) < 255.5, so the leading slice stays within +-255.
__device__ __forceinline__ int block_exp(float amax) {
  if (!(amax > 0.f)) return 0;
  int e;
  frexpf(amax, &e);
  if (KC > 64 && amax * pow2f(8 - e) >= 255.5f) ++e;
  return max(e, -90);  // keeps 2^(32-E) and 2^(E-16-8d) normal
}

// The NS integer slices of double-float values (hi, lo) for block exponent E, given s = 2^(8-E) and
// is = 2^(E-8) (all the powers of two involved are normal for the exponents block_exp returns),
// on two lanes with their own block factors: each step takes the integer of the leading plane,
// removes it exactly (FMA; the product is exact) and renormalises the remainder with the lo plane
// (TwoSum), so the slices carry the value to 2^-32 of the block whatever its size; the last
// slice is rounded to an integer.  The 16-bit codes are returned as (lane x, lane y) pairs.
// Every slice is an integer of magnitude at most 256, which keeps the two per-value conversions
// off the (quarter-rate) conversion pipe: the rounding to the nearest integer (ties to even) adds
// and removes 1.5 * 2^23 on packed FP32x2, exact for magnitudes below 2^22; and such an integer is
// exact in BF16, whose bits are then the upper half of the FP32 bits (one byte permutation packs
// the two lanes' codes).  FP16 codes come from the packed two-value conversion.
template <bool BF16, int NSL = NS>
__device__ __forceinline__ void slice_codes2_df(float2 vh, float2 vl, float2 s, float2 is,
                                                uint32_t (&code)[NSL]) {
  const float2 rnd = make_float2(12582912.f, 12582912.f), rnd_n = make_float2(-12582912.f, -12582912.f);
  float2 rh = vh, rl = vl, up = s, down = make_float2(-is.x, -is.y);
#pragma unroll
  for (int k = 0; k < NSL; ++k) {
    const float2 t = __fmul2_rn(rh, up);
    const float2 c = __fadd2_rn(__fadd2_rn(t, rnd), rnd_n);
    if (k + 1 < NSL) {
      const float2 h = __ffma2_rn(c, down, rh);
      two_sum2(h, rl, rh, rl);
    }
    up = mul2(256.f, up);
    down = mul2(0.00390625f, down);
    if (BF16) {
      code[k] = __byte_perm(__float_as_uint(c.x), __float_as_uint(c.y), 0x7632);
    } else {
      const __half2 h2 = __floats2half2_rn(c.x, c.y);
      code[k] = static_cast<uint32_t>(__half_as_ushort(__low2half(h2))) |
                (static_cast<uint32_t>(__half_as_ushort(__high2half(h2))) << 16);
    }
  }
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Column maxima of a warp's C x 32 block (v[i]: column i of this lane's row), by a transposing
// butterfly: at each step a lane keeps the half of its columns selected by its lane bit and takes
// the partner's copy of that half.  Returns, in lane l, the maximum over all 32 rows of column
// l mod C.  C - 1 exchanges instead of the C * 5 of one reduction per column.
template <int C>
__device__ __forceinline__ float column_max(float (&v)[C], int lane) {
  if (C == 16) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], __shfl_xor_sync(0xffffffffu, v[i], 16));
  }
#pragma unroll
  for (int w = C / 2; w >= 1; w /= 2) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float keep = up ? v[i + w] : v[i];
      const float give = up ? v[i] : v[i + w];
      v[i] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, give, w));
    }
  }
  return v[0];
}

__device__ __forceinline__ bool slot_runs(const SlotScalars* sc, int mode) {
  return mode == 0 ? sc->active != 0 : (mode == 1 ? sc->need_prec != 0 : true);
}

__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
}

struct TcStage {
  int M, N, K;
  void* out;        // next stage's slices, or nullptr in the last stage
  int8_t* eout;     // next stage's block exponents [N][M/64]
};

__device__ __forceinline__ TcStage tc_stage(const SlotDesc& S, int stage) {
  switch (stage) {
    case 0: return {S.nyp, S.nxp, S.nxp, S.tc_t1, S.tc_e[1]};
    case 1: return {S.nxp, S.nyp, S.nyp, S.tc_t2, S.tc_e[2]};
    case 2: return {S.nyp, S.nxp, S.nxp, S.tc_t3, S.tc_e[3]};
    default: return {S.nxp, S.nyp, S.nyp, nullptr, nullptr};
  }
}

template <bool BF16, int STAGE>
__global__ void __maxnreg__(kMaxRegs)
k_prec_tc(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
          const int* __restrict__ n_items, int mode, int* __restrict__ err, long long wait_cycles) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + STAGES * STAGE_BYTES);
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = *n_items;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int a = 0; a < kChunks; ++a) {
      mbar_init(&ctl->tfull[a], 1);
      mbar_init(&ctl->tempty[a], kEpiWarps);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = ctl->tmem;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0, issued = 0;
      uint32_t phase = 0;
      for (int w = blockIdx.x; w < total && !*abort_flag; w += gridDim.x) {
        const WorkItem it = items[w];
        const SlotDesc& S = slots[it.slot];
        if (!slot_runs(S.sc, mode)) continue;
        const TcStage v = tc_stage(S, STAGE);
        const void* ma = static_cast<const unsigned char*>(S.tmaps) + 128 * STAGE;
        const void* mb = static_cast<const unsigned char*>(S.tmaps) + 128 * (4 + STAGE);
        tmap_acquire(ma);
        tmap_acquire(mb);
        const int mt = v.M / BM;
        const int m0 = (it.tile % mt) * BM, n0 = (it.tile / mt) * BN;
        for (int kb = 0; kb < v.K / BK; ++kb) {
          if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_flag, wait_cycles)) break;
          mbar_expect_tx(&ctl->full[stage], STAGE_BYTES);
          unsigned char* sa = smem + stage * STAGE_BYTES;
          unsigned char* sb = sa + NS * A_PLANE;
#pragma unroll
          for (int p = 0; p < NS; ++p) tma_load_2d(sa + p * A_PLANE, ma, &ctl->full[stage], kb * BK, p * v.M + m0);
#pragma unroll
          for (int p = 0; p < NS; ++p) tma_load_2d(sb + p * B_PLANE, mb, &ctl->full[stage], kb * BK, p * v.N + n0);
          ++issued;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (*abort_flag) {
        // let the copies already issued (at most one per ring slot) land before the CTA leaves
        int s = stage;
        uint32_t ph = phase;
        for (int k = 0; k < STAGES && k < issued; ++k) {
          if (s == 0) {
            s = STAGES - 1;
            ph ^= 1;
          } else {
            --s;
          }
          const long long t0 = clock64();
          while (!mbar_try(&ctl->full[s], ph) && clock64() - t0 < kWaitCycles / 4) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0, chunk = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
        const WorkItem it = items[w];
        const SlotDesc& S = slots[it.slot];
        if (!slot_runs(S.sc, mode)) continue;
        const TcStage v = tc_stage(S, STAGE);
        for (int kb = 0; kb < v.K / BK; ++kb) {
          const int half_kb = kb % KPC;  // position inside the accumulation block
          const int cb = chunk % kChunks;
          if ((half_kb == 0 &&
               !mbar_wait(&ctl->tempty[cb], ((chunk / kChunks) & 1) ^ 1, abort_flag, wait_cycles)) ||
              !mbar_wait(&ctl->full[stage], phase, abort_flag, wait_cycles)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dset = tmem_base + cb * kSetCols;
          const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
          const uint32_t sb = sa + NS * A_PLANE;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
#pragma unroll
            for (int pa = 0; pa < NS; ++pa) {
              // slice pa of A against the B slices 0 .. NS-1-pa stacked along N (adjacent in
              // shared memory): one MMA adds A_pa B_pb to the accumulator of order pa + pb for
              // every pb, since the order accumulators are adjacent in TMEM the same way
              const uint64_t ad = sdesc(sa + pa * A_PLANE) + 2 * j;
              const uint64_t bd = sdesc(sb) + 2 * j;
              // the first MMA of an accumulation block (pa = 0) starts all NS orders afresh
              umma(dset + pa * BN, ad, bd, idesc_f16(BF16, BM, (NS - pa) * BN),
                   (half_kb > 0 || j > 0 || pa > 0) ? 1u : 0u);
            }
          }
          umma_commit(&ctl->empty[stage]);
          if (half_kb == KPC - 1) {
            umma_commit(&ctl->tfull[cb]);
            ++chunk;
          }
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // all MMAs issued by this thread complete before TMEM can be released
      umma_commit(&ctl->drain);
      const long long t0 = clock64();
      while (!mbar_try(&ctl->drain, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ epilogue
    const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
    const int group = (warp - 2) >> 2;       // columns kEpiCols*group .. +kEpiCols-1 of the tile
    const int ew = warp - 2;
    const int row = quarter * 32 + lane;
    const bool col_lane = lane < kEpiCols;   // lanes that own one of the warp's columns
    int chunk = 0;
    for (int w = blockIdx.x; w < total && !*abort_flag; w += gridDim.x) {
      const WorkItem it = items[w];
      const SlotDesc& S = slots[it.slot];
      SlotScalars* sc = S.sc;
      if (!slot_runs(sc, mode)) continue;
      const TcStage v = tc_stage(S, STAGE);
      const int mt = v.M / BM;
      const int m0 = (it.tile % mt) * BM, n0 = (it.tile / mt) * BN;
      const int m = m0 + row;
      const int ncol0 = n0 + group * kEpiCols;
      const int kblocks = v.K / KC;
      if (STAGE == 3 && col_lane && !S.mir_out) {
        // the r, q and mask entries read after the last k-block: start them towards L2 now
        const int n = ncol0 + lane;
        const int mr = min(m0 + 32 * quarter, S.nx - 1);
        if (n < S.ny && m0 + 32 * quarter < S.nx) {
          const size_t g = static_cast<size_t>(n) * S.nx + mr;
          const size_t g1 = static_cast<size_t>(n) * S.nx + min(mr + 31, S.nx - 1);
          asm volatile("prefetch.global.L2 [%0];" ::"l"(S.r + g));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(S.r + g1));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(S.q + g));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(S.q + g1));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(S.mask + g));
        }
      }
      // stage 1's eigenvalues, read now so their latency hides behind the k-blocks
      // and everything else the weights read from the descriptor, so that nothing is loaded after
      // the k-blocks: the row's flags, and per column lane a flag word (bit 0: the column is in the
      // grid, bit 1: it is in the low-mode block) that the weight loop takes by shuffles
      float lamx_m = 0.f, lamy_mine = 0.f, wnorm = 0.f;
      bool row_in = false, row_low = false;
      uint32_t col_flags = 0;
      if (STAGE == 1) {
        // issued here, not where the compiler would sink them: the MMA waits hide their latency
        row_in = m < S.nx;
        row_low = m < S.lowm_x;
        if (row_in) lamx_m = ld_early(S.lamx + m);
        const int n_mine = ncol0 + lane;
        if (col_lane && n_mine < S.ny) {
          lamy_mine = ld_early(S.lamy + n_mine);
          col_flags = 1u | (n_mine < S.lowm_y ? 2u : 0u);
        }
        wnorm = ld_early(&S.wnorm);
      }
      const int8_t* ea_row = S.tc_e[STAGE] + static_cast<size_t>(m) * kblocks;
      const int8_t* eb_col = S.tc_eb[STAGE] + static_cast<size_t>(ncol0 + (col_lane ? lane : 0)) * kblocks;
      // compensated (hi, lo) pairs of the warp's columns, two columns per packed register pair
      float2 hi[kEpiCols / 2], lo[kEpiCols / 2];
#pragma unroll
      for (int i = 0; i < kEpiCols / 2; ++i) {
        hi[i] = make_float2(0.f, 0.f);
        lo[i] = make_float2(0.f, 0.f);
      }
      bool fail_all = false;
      for (int kb = 0; kb < kblocks; ++kb) {
        const int cb = chunk % kChunks;
        // scale of the block sums: 2^(E_A + E_B - 16), as an exact product of two powers of two
        const float sa = pow2f(static_cast<int>(ea_row[kb]) - 16);
        const float sb_mine = pow2f(eb_col[kb]);
        // all epilogue warps leave together if any of them gave up waiting
        const uint32_t fail =
            mbar_wait(&ctl->tfull[cb], (chunk / kChunks) & 1, abort_flag, wait_cycles) ? 0u : 1u;
        uint32_t any_fail;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\t"
            "setp.ne.u32 p, %1, 0;\n\t"
            "bar.red.or.pred q, 1, %2, p;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(any_fail)
            : "r"(fail), "r"(32 * kEpiWarps)
            : "memory");
        if (any_fail) {
          fail_all = true;
          break;
        }
        tc_fence_after();
        const uint32_t base =
            tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + cb * kSetCols + group * kEpiCols;
#pragma unroll
        for (int hc = 0; hc < kEpiCols / kLdCols; ++hc) {
          uint32_t s0[kLdCols], s1[kLdCols], s2[kLdCols], s3[kLdCols];
          tmem_ld<kLdCols>(base + hc * kLdCols, s0);
          tmem_ld<kLdCols>(base + BN + hc * kLdCols, s1);
          tmem_ld<kLdCols>(base + 2 * BN + hc * kLdCols, s2);
          tmem_ld<kLdCols>(base + 3 * BN + hc * kLdCols, s3);
          tmem_wait_ld();
          if (hc == kEpiCols / kLdCols - 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->tempty[cb]);
          }
          // two columns per step on packed FP32x2; per column the operations and their order
          // are those of the scalar merge
          const float2 q8 = make_float2(0.00390625f, 0.00390625f);
#pragma unroll
          for (int i = 0; i < kLdCols; i += 2) {
            const int c = hc * kLdCols + i;
            const float2 scl = mul2(sa, make_float2(__shfl_sync(0xffffffffu, sb_mine, c),
                                                    __shfl_sync(0xffffffffu, sb_mine, c + 1)));
            const float2 v0 = make_float2(__uint_as_float(s0[i]), __uint_as_float(s0[i + 1]));
            const float2 v1 = make_float2(__uint_as_float(s1[i]), __uint_as_float(s1[i + 1]));
            const float2 v2 = make_float2(__uint_as_float(s2[i]), __uint_as_float(s2[i + 1]));
            const float2 v3 = make_float2(__uint_as_float(s3[i]), __uint_as_float(s3[i + 1]));
            // orders 1..3 combined first: their roundings are 2^-24 of terms 2^-8 below hi
            const float2 w = __ffma2_rn(v3, q8, v2);
            const float2 u = __ffma2_rn(w, q8, v1);
            const float2 t0 = __fmul2_rn(v0, scl);
            const float2 t1 = __fmul2_rn(u, __fmul2_rn(scl, q8));
            float2 er;
            two_sum2(hi[c / 2], t0, hi[c / 2], er);
            lo[c / 2] = add2(lo[c / 2], add2(er, t1));
          }
        }
        ++chunk;
      }
      if (fail_all) break;
      // the column sums as normalised double-float pairs (val, vlo)
      float val[kEpiCols], vlo[kEpiCols];
#pragma unroll
      for (int i = 0; i < kEpiCols / 2; ++i) {
        const f2x2 v = df_norm2(hi[i], lo[i]);
        val[2 * i] = v.hi.x;
        val[2 * i + 1] = v.hi.y;
        vlo[2 * i] = v.lo.x;
        vlo[2 * i + 1] = v.lo.y;
      }
      if (STAGE == 1) {
        // weight 1/(lam_y + lam_x)^2 (normalised); lam_y of the warp's columns via shuffles
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) {
          const float s = __shfl_sync(0xffffffffu, lamy_mine, i) + lamx_m;
          const uint32_t f = __shfl_sync(0xffffffffu, col_flags, i);
          // the low block (m < lowm_x, n < lowm_y) comes from the six-slice products instead
          const bool ok = row_in && (f & 1u) && (s > 0.f) && !(row_low && (f & 2u));
          const f2 wv = df_mul(f2{val[i], vlo[i]}, spectral_weight_of(wnorm, s));
          val[i] = ok ? wv.hi : 0.f;
          vlo[i] = ok ? wv.lo : 0.f;
        }
      }
      if (STAGE <= 2) {
        // block exponents of the next operand: rows n, k-blocks of KC consecutive m (lane quarters
        // 32q .. 32q+31 of this tile; KC/32 quarters per block, KC <= BM)
        float av[kEpiCols];
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) av[i] = fabsf(val[i]);
        const float mine = column_max<kEpiCols>(av, lane);
        if (col_lane) ctl->colmax[group][quarter][lane] = mine;
        epi_bar();
        float bmax = 0.f;
        const int q0 = (quarter / (KC / 32)) * (KC / 32);
        if (col_lane) {
#pragma unroll
          for (int q = 0; q < KC / 32; ++q) bmax = fmaxf(bmax, ctl->colmax[group][q0 + q][lane]);
        }
        const int E_mine = block_exp(bmax);
        const float s_mine = pow2f(8 - E_mine), is_mine = pow2f(E_mine - 8);
        // no second barrier before colmax is rewritten: that happens after the next tile's first
        // k-block, whose failure vote every epilogue warp joins only after these reads
        const size_t plane = static_cast<size_t>(v.M) * v.N;
        uint16_t* out = static_cast<uint16_t*>(v.out);
#pragma unroll
        for (int i = 0; i < kEpiCols; i += 2) {
          const float2 s2 = make_float2(__shfl_sync(0xffffffffu, s_mine, i), __shfl_sync(0xffffffffu, s_mine, i + 1));
          const float2 is2 =
              make_float2(__shfl_sync(0xffffffffu, is_mine, i), __shfl_sync(0xffffffffu, is_mine, i + 1));
          uint32_t code[NS];
          slice_codes2_df<BF16>(make_float2(val[i], val[i + 1]), make_float2(vlo[i], vlo[i + 1]), s2,
                                is2, code);
          const size_t i0 = static_cast<size_t>(ncol0 + i) * v.M + m, i1 = i0 + v.M;
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            out[q * plane + i0] = static_cast<uint16_t>(code[q] & 0xffffu);
            out[q * plane + i1] = static_cast<uint16_t>(code[q] >> 16);
          }
        }
        if (quarter == q0 && col_lane)
          v.eout[static_cast<size_t>(ncol0 + lane) * (v.M / KC) + (m0 + 32 * quarter) / KC] =
              static_cast<int8_t>(E_mine);
      } else {
        CompDotDF c_rz, c_zq;
        const bool with_zq = S.mir_out == 0 && (sc->flexible != 0 || mode == 2);
        if (m < S.nx) {
          constexpr int kGrp = 8;
          static_assert(kEpiCols % kGrp == 0, "stage-3 load groups");
#pragma unroll
          for (int g8 = 0; g8 < kEpiCols; g8 += kGrp) {
            if (S.lowm_x) {
              // the low-mode part first: the 32-bit stages' result plus zl, one double-float value
              const size_t nn = static_cast<size_t>(S.nx) * S.ny;
              float wh[kGrp], wl[kGrp];
#pragma unroll
              for (int i = 0; i < kGrp; ++i) {
                const int n = ncol0 + g8 + i;
                const size_t g = static_cast<size_t>(n < S.ny ? n : 0) * S.nx + m;
                wh[i] = S.low_z[g];
                wl[i] = S.low_z[nn + g];
              }
#pragma unroll
              for (int i = 0; i < kGrp; ++i) {
                const f2 zsum = df_add(f2{val[g8 + i], vlo[g8 + i]}, f2{wh[i], wl[i]});
                val[g8 + i] = zsum.hi;
                vlo[g8 + i] = zsum.lo;
              }
            }
            if (S.mir_out) {
              // one mirror class of a folded slot: its result g, unmasked (k_unfold combines the
              // classes, masks and forms the dot products)
#pragma unroll
              for (int i = 0; i < kGrp; ++i) {
                const int n = ncol0 + g8 + i;
                if (n < S.ny) {
                  S.z[n * S.nx + m] = val[g8 + i];
                  S.z_lo[n * S.nx + m] = vlo[g8 + i];
                }
              }
              continue;
            }
            float rv[kGrp], rl[kGrp], qv[kGrp], ql[kGrp];
            uint8_t mk[kGrp];
#pragma unroll
            for (int i = 0; i < kGrp; ++i) {  // issue the group's loads together
              const int n = ncol0 + g8 + i;
              const int g = (n < S.ny ? n : 0) * S.nx + m;
              rv[i] = S.r[g];
              rl[i] = S.r_lo[g];
              // z.q enters only the flexible beta
              qv[i] = with_zq ? S.q[g] : 0.f;
              ql[i] = with_zq ? S.q_lo[g] : 0.f;
              mk[i] = n < S.ny ? S.mask[g] : 0;
            }
#pragma unroll
            for (int i = 0; i < kGrp; ++i) {
              const int n = ncol0 + g8 + i;
              if (n < S.ny) {
                const float zh = mk[i] ? val[g8 + i] : 0.f;
                const float zl = mk[i] ? vlo[g8 + i] : 0.f;
                S.z[n * S.nx + m] = zh;
                S.z_lo[n * S.nx + m] = zl;
                c_rz.add(rv[i], rl[i], zh, zl);
                c_zq.add(zh, zl, qv[i], ql[i]);
              }
            }
          }
        }
        if (S.mir_out) continue;  // a class problem leaves no partial sums
        // tile partials of r.z and z.q (FP32-compensated inside the warp)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          float e;
          const float a1 = __shfl_xor_sync(0xffffffffu, c_rz.s, o), a2 = __shfl_xor_sync(0xffffffffu, c_rz.c, o);
          two_sum(c_rz.s, a1, c_rz.s, e);
          c_rz.c = __fadd_rn(c_rz.c, __fadd_rn(a2, e));
          const float b1 = __shfl_xor_sync(0xffffffffu, c_zq.s, o), b2 = __shfl_xor_sync(0xffffffffu, c_zq.c, o);
          two_sum(c_zq.s, b1, c_zq.s, e);
          c_zq.c = __fadd_rn(c_zq.c, __fadd_rn(b2, e));
        }
        if (lane == 0) {
          ctl->red[ew][0] = c_rz.s;
          ctl->red[ew][1] = c_rz.c;
          ctl->red[ew][2] = c_zq.s;
          ctl->red[ew][3] = c_zq.c;
        }
        epi_bar();
        if (ew == 0) {
          // the warps' compensated pairs, summed the same way across lanes 0 .. kEpiWarps-1
          CompDot t_rz, t_zq;
          if (lane < kEpiWarps) {
            t_rz.s = ctl->red[lane][0];
            t_rz.c = ctl->red[lane][1];
            t_zq.s = ctl->red[lane][2];
            t_zq.c = ctl->red[lane][3];
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            float e;
            const float a1 = __shfl_xor_sync(0xffffffffu, t_rz.s, o), a2 = __shfl_xor_sync(0xffffffffu, t_rz.c, o);
            two_sum(t_rz.s, a1, t_rz.s, e);
            t_rz.c = __fadd_rn(t_rz.c, __fadd_rn(a2, e));
            const float b1 = __shfl_xor_sync(0xffffffffu, t_zq.s, o), b2 = __shfl_xor_sync(0xffffffffu, t_zq.c, o);
            two_sum(t_zq.s, b1, t_zq.s, e);
            t_zq.c = __fadd_rn(t_zq.c, __fadd_rn(b2, e));
          }
          // tile partials; k_prec_finish forms rho and beta from them
          if (lane == 0) {
            S.part[it.tile * 4 + 2] = t_rz.value();
            S.part[it.tile * 4 + 3] = t_zq.value();
          }
        }
        // ctl->red is rewritten only after the next tile's first k-block (see stages 0..2)
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0 && ctl->abort_flag) atomicExch(err, 1);
}

// Residual -> slices of the first stage's A operand (slots with no folded axis).  One item per
// 32 rows and KC columns; one warp per four of the rows, all four loaded before any is sliced.
template <bool BF16>
__global__ void __launch_bounds__(256)
k_tc_prepare(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
             const int* __restrict__ n_items, int mode) {
  const int total = *n_items;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    if (!slot_runs(sc, mode) || S.mir) continue;  // folded slots: k_tc_fold
    const int tx = (S.nx + KC - 1) / KC;
    const int x0 = (it.tile % tx) * KC;
    const int y0 = (it.tile / tx) * kStTileY;
    const int kblocks = S.nxp / KC;
    const size_t plane = static_cast<size_t>(S.nyp) * S.nxp;
    uint16_t* out = static_cast<uint16_t*>(S.tc_r);
    // every row of the warp loaded before any is sliced
    constexpr int kRows = kStTileY / 8;
    static_assert(kRows * 8 == kStTileY, "rows per warp");
    // each lane takes adjacent pairs (x, x+1) and writes both codes of a slice in one 4-byte
    // store (x even, rows of nxp even: aligned)
    constexpr int kPairs = KC / 64;
    float2 v[kRows][kPairs], vl[kRows][kPairs];
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const int y = y0 + warp + 8 * j;
#pragma unroll
      for (int k = 0; k < kPairs; ++k) {
        const int x = x0 + 64 * k + 2 * lane;
        const float* row = S.r + static_cast<size_t>(y) * S.nx;
        const float* row_lo = S.r_lo + static_cast<size_t>(y) * S.nx;
        v[j][k].x = (x < S.nx && y < S.ny) ? row[x] : 0.f;
        v[j][k].y = (x + 1 < S.nx && y < S.ny) ? row[x + 1] : 0.f;
        vl[j][k].x = (x < S.nx && y < S.ny) ? row_lo[x] : 0.f;
        vl[j][k].y = (x + 1 < S.nx && y < S.ny) ? row_lo[x + 1] : 0.f;
      }
    }
    uint32_t* out32 = reinterpret_cast<uint32_t*>(out);
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const int y = y0 + warp + 8 * j;
      if (y >= S.ny) break;
      float amax = 0.f;
#pragma unroll
      for (int k = 0; k < kPairs; ++k) amax = fmaxf(amax, fmaxf(fabsf(v[j][k].x), fabsf(v[j][k].y)));
      const int E = block_exp(warp_max(amax));
      const float s = pow2f(8 - E), is = pow2f(E - 8);
#pragma unroll
      for (int k = 0; k < kPairs; ++k) {
        const size_t idx = (static_cast<size_t>(y) * S.nxp + x0 + 64 * k + 2 * lane) / 2;
        if (S.lowm_x) {
          // six slices: the first four are stage 0's operand, all six the low-mode product's
          uint32_t code[kLowNS];
          slice_codes2_df<BF16, kLowNS>(v[j][k], vl[j][k], make_float2(s, s), make_float2(is, is), code);
#pragma unroll
          for (int q = 0; q < kLowNS; ++q) out32[q * (plane / 2) + idx] = code[q];
        } else {
          uint32_t code[NS];
          slice_codes2_df<BF16, NS>(v[j][k], vl[j][k], make_float2(s, s), make_float2(is, is), code);
#pragma unroll
          for (int q = 0; q < NS; ++q) out32[q * (plane / 2) + idx] = code[q];
        }
      }
      if (lane == 0) S.tc_e[0][static_cast<size_t>(y) * kblocks + x0 / KC] = static_cast<int8_t>(E);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Mirror fold (slots with a folded axis).  On a folded axis the basis splits into even and odd
// vectors under i -> n-1-i (plan.cpp), so the four stages of the slot run as two or four
// independent half-size problems, its classes.  k_tc_fold forms each class's residual on its
// ceil(n/2)-node domain, signed sums of r at a node and its mirrors (the even class adds, the
// odd class subtracts; a middle node, its own mirror, counts once in the even class and not in
// the odd one), in double-float, and slices it like k_tc_prepare.  After stage 3 has written
// each class's result g, k_unfold forms z at a node and its mirrors as the sums of the classes
// with the odd ones' signs flipped on the mirrored side, masks it and leaves the r.z and z.q
// partials that stage 3 leaves for an unfolded slot.
// ---------------------------------------------------------------------------------------------

// One warp per (class row y, 128 class columns); lane pairs (x, x+1) at x = 64 k + 2 lane.
template <bool BF16>
__global__ void __launch_bounds__(256, 4)
k_tc_fold(const SlotDesc* __restrict__ slots, const SlotDesc* __restrict__ tcp,
          const WorkItem* __restrict__ items, const int* __restrict__ n_items, int mode) {
  const int total = *n_items;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    if (!slot_runs(S.sc, mode)) continue;
    const bool fx = (S.mir & 1) != 0, fy = (S.mir & 2) != 0;
    const int nxb = (S.mhx + KC - 1) / KC;
    const int y = (it.tile / nxb) * 8 + warp, xb = it.tile % nxb;
    if (y >= S.mhy) continue;
    const int yy = fy ? S.ny - 1 - y : y;  // the mirrored row (y itself on an unfolded axis)
    const bool ymid = yy == y;
    const float* rh = S.r;
    const float* rl = S.r_lo;
    // class values of the lane's four columns: hi and lo planes of pair k's columns (x, x+1)
    float2 ch[4][2], cl[4][2];  // [class][pair]
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      f2 v[4][2];  // [class][column of the pair]
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int x = xb * KC + 64 * k + 2 * lane + e;
        f2 a{0.f, 0.f}, b{0.f, 0.f}, c{0.f, 0.f}, d{0.f, 0.f};
        const int xx = fx ? S.nx - 1 - x : x;
        const bool xmid = xx == x;
        if (x < S.mhx) {
          const size_t gy = static_cast<size_t>(y) * S.nx, gyy = static_cast<size_t>(yy) * S.nx;
          a = f2{rh[gy + x], rl[gy + x]};
          if (!xmid) b = f2{rh[gy + xx], rl[gy + xx]};
          if (!ymid) {
            c = f2{rh[gyy + x], rl[gyy + x]};
            if (!xmid) d = f2{rh[gyy + xx], rl[gyy + xx]};
          }
        }
        // along x: even = a + b, odd = a - b (b = 0 at a middle node or on an unfolded axis)
        const f2 e0 = df_add(a, b), o0 = df_add(a, df_neg(b));
        const f2 e1 = df_add(c, d), o1 = df_add(c, df_neg(d));
        // along y the same with the mirrored row; class c = 2 cls_y + cls_x
        v[0][e] = df_add(e0, e1);
        v[1][e] = df_add(o0, o1);
        v[2][e] = df_add(e0, df_neg(e1));
        v[3][e] = df_add(o0, df_neg(o1));
        if (xmid && fx) {  // the odd x classes vanish at the middle column
          v[1][e] = f2{0.f, 0.f};
          v[3][e] = f2{0.f, 0.f};
        }
        if (ymid && fy) {
          v[2][e] = f2{0.f, 0.f};
          v[3][e] = f2{0.f, 0.f};
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        ch[c][k] = make_float2(v[c][0].hi, v[c][1].hi);
        cl[c][k] = make_float2(v[c][0].lo, v[c][1].lo);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if ((c & 1) && !fx) continue;
      if ((c & 2) && !fy) continue;
      const SlotDesc& T = tcp[kMirClasses * it.slot + c];
      float amax = 0.f;
#pragma unroll
      for (int k = 0; k < 2; ++k) amax = fmaxf(amax, fmaxf(fabsf(ch[c][k].x), fabsf(ch[c][k].y)));
      const int E = block_exp(warp_max(amax));
      const float up = pow2f(8 - E), is = pow2f(E - 8);
      const size_t plane = static_cast<size_t>(T.nyp) * T.nxp;
      uint32_t* out32 = static_cast<uint32_t*>(T.tc_r);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const size_t idx = (static_cast<size_t>(y) * T.nxp + xb * KC + 64 * k + 2 * lane) / 2;
        if (T.lowm_x) {
          uint32_t code[kLowNS];
          slice_codes2_df<BF16, kLowNS>(ch[c][k], cl[c][k], make_float2(up, up), make_float2(is, is), code);
#pragma unroll
          for (int q = 0; q < kLowNS; ++q) out32[q * (plane / 2) + idx] = code[q];
        } else {
          uint32_t code[NS];
          slice_codes2_df<BF16, NS>(ch[c][k], cl[c][k], make_float2(up, up), make_float2(is, is), code);
#pragma unroll
          for (int q = 0; q < NS; ++q) out32[q * (plane / 2) + idx] = code[q];
        }
      }
      if (lane == 0) T.tc_e[0][static_cast<size_t>(y) * (T.nxp / KC) + xb] = static_cast<int8_t>(E);
    }
  }
}

// One thread per class node (tiles of 32 x 8): z at the node and its mirrors, masked, with the
// tile's compensated r.z and z.q partials.
__global__ void __launch_bounds__(256)
k_unfold(const SlotDesc* __restrict__ slots, const SlotDesc* __restrict__ tcp,
         const WorkItem* __restrict__ items, const int* __restrict__ n_items, int mode) {
  __shared__ float red[8][4];
  const int total = *n_items;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    if (!slot_runs(S.sc, mode)) continue;
    const bool fx = (S.mir & 1) != 0, fy = (S.mir & 2) != 0;
    const int ntx = (S.mhx + 31) >> 5;
    const int x = (it.tile % ntx) * 32 + lane, y = (it.tile / ntx) * 8 + warp;
    CompDotDF c_rz, c_zq;
    const bool with_zq = S.sc->flexible != 0 || mode == 2;  // z.q enters only the flexible beta
    if (x < S.mhx && y < S.mhy) {
      const int xx = fx ? S.nx - 1 - x : x, yy = fy ? S.ny - 1 - y : y;
      // every load first: the classes' g at (y, x), then mask, r (and q) at the mirror nodes
      f2 g[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        g[c] = f2{0.f, 0.f};
        if (((c & 1) && !fx) || ((c & 2) && !fy)) continue;
        const SlotDesc& T = tcp[kMirClasses * it.slot + c];
        const int gi = y * T.nx + x;
        g[c] = f2{T.z[gi], T.z_lo[gi]};
      }
      int gi[4];
      bool live[4];
      uint8_t mk[4];
      float rh[4], rl[4], qh[4], ql[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {  // t = 2 (mirrored row) + (mirrored column)
        live[t] = !((t & 1) && xx == x) && !((t & 2) && yy == y);
        gi[t] = ((t & 2) ? yy : y) * S.nx + ((t & 1) ? xx : x);
        mk[t] = 0;
        rh[t] = rl[t] = qh[t] = ql[t] = 0.f;
        if (live[t]) {
          mk[t] = S.mask[gi[t]];
          rh[t] = S.r[gi[t]];
          rl[t] = S.r_lo[gi[t]];
          if (with_zq) {
            qh[t] = S.q[gi[t]];
            ql[t] = S.q_lo[gi[t]];
          }
        }
      }
      // even/odd butterflies along x, then y
      const f2 a = df_add(g[0], g[1]), b = df_add(g[0], df_neg(g[1]));
      const f2 c = df_add(g[2], g[3]), d = df_add(g[2], df_neg(g[3]));
      const f2 v[4] = {df_add(a, c), df_add(b, d), df_add(a, df_neg(c)), df_add(b, df_neg(d))};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (!live[t]) continue;
        const float zh = mk[t] ? v[t].hi : 0.f, zl = mk[t] ? v[t].lo : 0.f;
        S.z[gi[t]] = zh;
        S.z_lo[gi[t]] = zl;
        c_rz.add(rh[t], rl[t], zh, zl);
        if (with_zq) c_zq.add(zh, zl, qh[t], ql[t]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float e;
      const float a1 = __shfl_xor_sync(0xffffffffu, c_rz.s, o), a2 = __shfl_xor_sync(0xffffffffu, c_rz.c, o);
      two_sum(c_rz.s, a1, c_rz.s, e);
      c_rz.c = __fadd_rn(c_rz.c, __fadd_rn(a2, e));
      const float b1 = __shfl_xor_sync(0xffffffffu, c_zq.s, o), b2 = __shfl_xor_sync(0xffffffffu, c_zq.c, o);
      two_sum(c_zq.s, b1, c_zq.s, e);
      c_zq.c = __fadd_rn(c_zq.c, __fadd_rn(b2, e));
    }
    if (lane == 0) {
      red[warp][0] = c_rz.s;
      red[warp][1] = c_rz.c;
      red[warp][2] = c_zq.s;
      red[warp][3] = c_zq.c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      CompDot t_rz, t_zq;
      for (int k = 0; k < 8; ++k) {  // the warps in order
        float e;
        two_sum(t_rz.s, red[k][0], t_rz.s, e);
        t_rz.c = __fadd_rn(t_rz.c, __fadd_rn(red[k][1], e));
        two_sum(t_zq.s, red[k][2], t_zq.s, e);
        t_zq.c = __fadd_rn(t_zq.c, __fadd_rn(red[k][3], e));
      }
      S.part[it.tile * 4 + 2] = t_rz.value();
      S.part[it.tile * 4 + 3] = t_zq.value();
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Low-mode correction (mixed modes).  The weights 1/(lam_y + lam_x)^2 of the smoothest modes are up
// to (64/lam_min)^2 times those of the roughest, so rounding noise of the 32-bit stages, relative
// to |r|, is amplified in exactly these modes and costs CG iterations.  The modes kx < 32,
// ky < 32 (of each transform problem) are therefore left out of stage 1's weights and computed
// here to about 48 bits:
//   forward (k_low_tc):  H[y][kx] = sum_x r[y][x] Qx[x][kx], six slices each side, and each
//                        128-row tile's share of G = Qy_low^T H (double-float dot products)
//   middle (k_low_mid):  G = the shares in tile order, G' = w o G,
//                        J[ky][x] = sum_kx G'[ky][kx] Qx[x][kx] (double-float), J^T in six slices
//   inverse (k_low_inv): zl[y][x] = sum_ky Qy[y][ky] J[ky][x], six slices each side
// and stage 3 adds zl to its result.  With six 8-bit slices per operand the products of orders
// 0..5 (21 of them) are kept, each order in its own TMEM accumulator; per k, the products of one
// order add up to at most 2^17 in magnitude, so over a 128-wide block every partial sum is an
// exact integer of at most 2^24.  Orders 0..2 are merged into the double-float result with TwoSum,
// orders 3..5 (below 2^-24 of it) in plain FP32.
//
// The forward product: one CTA per 128 rows of y, sixteen warps (four per TMEM lane quarter, eight
// of the 32 columns each); thread 0 issues the tensor copies and the MMAs one 64-wide k step at a
// time (the products are thin, so a simple serial pipeline suffices), every thread drains its own
// TMEM lane after each exponent block, and after the last block the CTA forms its share of G.
// ---------------------------------------------------------------------------------------------
constexpr int LBN = kLowM;                   // N tile (columns)
constexpr int LBK = 64;                      // k per tensor copy
constexpr int LA_PLANE = BM * LBK * 2;       // 16 KB
constexpr int LB_PLANE = LBN * LBK * 2;      // 4 KB
constexpr int kLowThreads = 512;              // 16 warps: four per TMEM lane quarter
constexpr int kLowCols = LBN / 4;             // columns per warp in the merge
constexpr int kLowTmemCols = 256;            // >= kLowNS * LBN
constexpr int kLowSmem = kLowNS * (LA_PLANE + LB_PLANE) + 1024 + 256;
static_assert(kLowNS * LBN <= kLowTmemCols, "low-mode TMEM columns");
static_assert(kLowK3 == LBK, "the inverse product's k fits one copy");
static_assert(kLowThreads == 16 * 32 && 2 * BM * 33 * 4 + 2 * BM * kLowM * 4 <= kLowNS * (LA_PLANE + LB_PLANE),
              "the G stage: sixteen warps (ky = 2 warp, 2 warp + 1) and its staging in the operand buffers");
static_assert((2 * BM * 33) % 2 == 0 && kLowM % 2 == 0, "8-byte aligned Qy_low pairs in the G stage");
static_assert((BM * kLowM) % kLowThreads == 0, "the tile's Qy_low rows in equal shares per thread");

struct LowCtl {
  uint64_t full, done;
  uint32_t tmem;
  int abort_flag;
};

// Exponent of a block whose largest magnitude is amax: amax < 2^E and amax 2^(8-E) < 255.5.
__device__ __forceinline__ int low_block_exp(float amax) {
  if (!(amax > 0.f)) return 0;
  int e;
  frexpf(amax, &e);
  if (amax * pow2f(8 - e) >= 255.5f) ++e;
  return max(e, -90);
}

template <bool BF16>
__global__ void __launch_bounds__(kLowThreads, 1)
k_low_tc(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
         const int* __restrict__ n_items, int mode, int* __restrict__ err, long long wait_cycles) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  LowCtl* ctl = reinterpret_cast<LowCtl*>(smem + kLowNS * (LA_PLANE + LB_PLANE));
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = *n_items;
  if (threadIdx.x == 0) {
    mbar_init(&ctl->full, 1);
    mbar_init(&ctl->done, 1);
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem)),
                 "r"(kLowTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = ctl->tmem;
  uint32_t ph_full = 0, ph_done = 0;
  int inflight = 0;     // thread 0: tensor copies issued and not yet waited for (0 or 1)
  int mma_pending = 0;  // thread 0: MMAs committed and not yet waited for (0 or 1)
  const int quarter = warp & 3, cg = warp >> 2;  // TMEM lane quarter, column group
  const int row = quarter * 32 + lane;          // TMEM lane of this thread = tile row
  bool failed = false;
  for (int w = blockIdx.x; w < total && !failed; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    if (!slot_runs(S.sc, mode) || S.lowm_x == 0) continue;
    // geometry: A = the residual's six slice planes (rows y), B = Qx_low^T's (rows kx)
    const unsigned char* maps = static_cast<const unsigned char*>(S.low_maps);
    const void* ma = maps;
    const void* mb = maps + 128;
    const int m0 = it.tile * BM, n0 = 0, K = S.nxp, KC = 128, rowsA = S.nyp, rowsB = kLowM;
    if (threadIdx.x == 0) {
      tmap_acquire(ma);
      tmap_acquire(mb);
    }
    const int m = m0 + row;
    // the thread's share of the tile's Qy_low rows (the G stage's operand), loaded now so that
    // their latency hides behind the k-blocks
    constexpr int kYq = BM * kLowM / kLowThreads;
    float yq[2 * kYq];
#pragma unroll
    for (int i = 0; i < kYq; ++i) {
      const size_t a = static_cast<size_t>(m0) * kLowM + threadIdx.x + i * kLowThreads;
      yq[i] = ld_early(S.low_qyd + a);
      yq[kYq + i] = ld_early(S.low_qyd + static_cast<size_t>(S.nyp) * kLowM + a);
    }
    // double-float result of the thread's row, one per column of its group
    float hi[kLowCols], lo[kLowCols];
#pragma unroll
    for (int c = 0; c < kLowCols; ++c) {
      hi[c] = 0.f;
      lo[c] = 0.f;
    }
    for (int kb = 0; kb < K / KC && !failed; ++kb) {
      if (threadIdx.x == 0) {
        for (int sub = 0; sub < KC / LBK; ++sub) {
          const int k0 = kb * KC + sub * LBK;
          unsigned char* sa = smem;
          unsigned char* sb = smem + kLowNS * LA_PLANE;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(&ctl->full, kLowNS * (LA_PLANE + LB_PLANE));
#pragma unroll
          for (int p = 0; p < kLowNS; ++p) tma_load_2d(sa + p * LA_PLANE, ma, &ctl->full, k0, p * rowsA + m0);
#pragma unroll
          for (int p = 0; p < kLowNS; ++p) tma_load_2d(sb + p * LB_PLANE, mb, &ctl->full, k0, p * rowsB + n0);
          inflight = 1;
          if (!mbar_wait(&ctl->full, ph_full, abort_flag, wait_cycles)) break;
          inflight = 0;
          ph_full ^= 1;
          tc_fence_after();
          const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
          for (int j = 0; j < LBK / 16; ++j) {
#pragma unroll
            for (int i = 0; i < kLowNS; ++i) {
              // slice i of A against the B slices 0 .. kLowNS-1-i stacked along N: order i + j'
              // lands in the accumulator at column (i + j') * LBN
              umma(tmem_base + i * LBN, sdesc(a0 + i * LA_PLANE) + 2 * j, sdesc(b0) + 2 * j,
                   idesc_f16(BF16, BM, (kLowNS - i) * LBN), (sub > 0 || j > 0 || i > 0) ? 1u : 0u);
            }
          }
          umma_commit(&ctl->done);
          // the next copy reuses the shared memory, and the block's sums must be complete
          mma_pending = 1;
          if (!mbar_wait(&ctl->done, ph_done, abort_flag, wait_cycles)) break;
          mma_pending = 0;
          ph_done ^= 1;
        }
      }
      __syncthreads();
      if (*abort_flag) {
        failed = true;
        break;
      }
      tc_fence_after();
      // exponents of the block: the thread's row (A) and every column (B)
      const int ea = S.tc_e[0][static_cast<size_t>(min(m, S.nyp - 1)) * (S.nxp / 128) + kb];
      // 2^(E_A + E_B - 16) of every column (exact products of powers of two)
      float scl[kLowCols];
#pragma unroll
      for (int c = 0; c < kLowCols; ++c) {
        const int cc = cg * kLowCols + c;
        const int eb = S.low_qxt_e[static_cast<size_t>(cc) * (S.nxp / 128) + kb];
        scl[c] = pow2f(ea - 16) * pow2f(eb);
      }
      // the six order sums of the warp's columns, loaded together
      uint32_t v[kLowNS][kLowCols];
#pragma unroll
      for (int d = 0; d < kLowNS; ++d)
        tmem_ld8(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + d * LBN + cg * kLowCols, v[d]);
      tmem_wait_ld();
#pragma unroll
      for (int d = 0; d < kLowNS; ++d) {
        const float od = pow2f(-8 * d);
#pragma unroll
        for (int c = 0; c < kLowCols; ++c) {
          const float t = __uint_as_float(v[d][c]) * scl[c] * od;
          if (d <= 2) {
            float e;
            two_sum(hi[c], t, hi[c], e);
            lo[c] = __fadd_rn(lo[c], e);
          } else {
            lo[c] = __fadd_rn(lo[c], t);
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // the next block's MMAs overwrite the accumulators
    }
    if (failed) break;
    {
      // the tile's share of G = Qy_low^T H (its 128 rows of y), by compensated dot products of
      // double-float operands staged in shared memory (the operand buffers are free: the last
      // MMAs completed before the block's TMEM reads); H itself is not stored
      float* hs = reinterpret_cast<float*>(smem);  // H tile [128][33]: hi, then lo
      float* ys = hs + 2 * BM * 33;                 // Qy_low rows m0 .. m0+127 [128][32]: hi, lo
#pragma unroll
      for (int c = 0; c < kLowCols; ++c) {
        const f2 hv = df_norm(hi[c], lo[c]);
        hs[row * 33 + cg * kLowCols + c] = hv.hi;
        hs[BM * 33 + row * 33 + cg * kLowCols + c] = hv.lo;
      }
#pragma unroll
      for (int i = 0; i < kYq; ++i) {
        ys[threadIdx.x + i * kLowThreads] = yq[i];
        ys[BM * kLowM + threadIdx.x + i * kLowThreads] = yq[kYq + i];
      }
      __syncthreads();
      // thread: kx = lane, ky = 2 warp and 2 warp + 1, the two dot products on packed FP32x2
      // (one 8-byte broadcast load of each plane's Qy_low pair per row)
      CompDotDF2 g;
      const int ky0 = 2 * warp;
#pragma unroll 4
      for (int rr = 0; rr < BM; ++rr) {
        const float bh = hs[rr * 33 + lane], bl = hs[BM * 33 + rr * 33 + lane];
        const float2 ah = *reinterpret_cast<const float2*>(ys + rr * kLowM + ky0);
        const float2 al = *reinterpret_cast<const float2*>(ys + BM * kLowM + rr * kLowM + ky0);
        g.add(ah, al, make_float2(bh, bh), make_float2(bl, bl));
      }
      float* gp = S.low_gp + static_cast<size_t>(it.tile) * 2 * kLowM * kLowM;
      const f2 a0 = df_norm(g.s.x, g.c.x), a1 = df_norm(g.s.y, g.c.y);
      gp[ky0 * kLowM + lane] = a0.hi;
      gp[kLowM * kLowM + ky0 * kLowM + lane] = a0.lo;
      gp[(ky0 + 1) * kLowM + lane] = a1.hi;
      gp[kLowM * kLowM + (ky0 + 1) * kLowM + lane] = a1.lo;
      __syncthreads();  // the next item's tensor copies overwrite the staging
    }
  }
  if (threadIdx.x == 0) {
    // after an abort: a copy still in flight lands, and committed MMAs complete, before the CTA
    // frees its TMEM and leaves
    if (inflight) {
      const long long t0 = clock64();
      while (!mbar_try(&ctl->full, ph_full) && clock64() - t0 < kWaitCycles / 4) {
      }
    }
    if (mma_pending) {
      const long long t0 = clock64();
      while (!mbar_try(&ctl->done, ph_done) && clock64() - t0 < kWaitCycles / 4) {
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kLowTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0 && ctl->abort_flag) atomicExch(err, 1);
}

// Inverse low-mode product, zl[y][x] = sum_ky Qy[y][ky] J[ky][x], one item per (slot, 128-row
// tile of x).  The tile's six J^T slice planes (its A operand, k = ky padded to 64; the products
// use the 32 real k) are copied once; the B operand (Qy_low's slices for 32 values of y) is
// double-buffered, each copy issued two y-tiles ahead (as soon as the products that read its
// buffer are complete), and the products of consecutive y-tiles go to two TMEM sets, so that the
// MMAs of one y-tile run while the sixteen warps merge and store the previous one.
struct LowInvCtl {
  uint64_t fa, fb[2], md[2];
  uint32_t tmem;
  int abort_flag;
};
constexpr int kLowInvSmem = kLowNS * LA_PLANE + 2 * kLowNS * LB_PLANE + 1024 + 256;
constexpr int kLowInvThreads = 512;            // 16 warps: four per TMEM lane quarter
constexpr int kLowInvCols = LBN / 4;           // columns per warp
constexpr int kLowInvTmemCols = 512;  // two sets of kLowNS * LBN columns, at 0 and 256
static_assert(kLowNS * LBN <= 256, "low-mode TMEM set");

template <bool BF16>
__global__ void __launch_bounds__(kLowInvThreads, 1)
k_low_inv(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
          const int* __restrict__ n_items, int mode, int* __restrict__ err, long long wait_cycles) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* sA = smem;
  unsigned char* sB = smem + kLowNS * LA_PLANE;  // two buffers of kLowNS * LB_PLANE
  LowInvCtl* ctl = reinterpret_cast<LowInvCtl*>(sB + 2 * kLowNS * LB_PLANE);
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = *n_items;
  if (threadIdx.x == 0) {
    mbar_init(&ctl->fa, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->fb[b], 1);
      mbar_init(&ctl->md[b], 1);
    }
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem)),
                 "r"(kLowInvTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = ctl->tmem;
  // thread 0's barrier bookkeeping: phases and the waits still owed
  uint32_t ph_fa = 0, ph_fb[2] = {0, 0}, ph_md[2] = {0, 0};
  int owe_fa = 0, owe_fb[2] = {0, 0}, owe_md[2] = {0, 0};
  const int quarter = warp & 3, cg = warp >> 2;   // TMEM lane quarter, column group
  const int row = quarter * 32 + lane;
  bool failed = false;
  for (int w = blockIdx.x; w < total && !failed; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    if (!slot_runs(S.sc, mode) || S.lowm_x == 0) continue;
    const unsigned char* maps = static_cast<const unsigned char*>(S.low_maps);
    const void* ma = maps + 128 * 2;
    const void* mb = maps + 128 * 3;
    const int m0 = it.tile * BM;
    const int nt = S.nyp / LBN;
    auto issue_b = [&](int j) {  // thread 0: B slices of y-tile j into buffer j & 1
      const int b = j & 1;
      unsigned char* dst = sB + b * kLowNS * LB_PLANE;
      mbar_expect_tx(&ctl->fb[b], kLowNS * LB_PLANE);
#pragma unroll
      for (int p = 0; p < kLowNS; ++p) tma_load_2d(dst + p * LB_PLANE, mb, &ctl->fb[b], 0, p * S.nyp + j * LBN);
      owe_fb[b] = 1;
    };
    auto issue_mma = [&](int j) -> bool {  // thread 0: wait for B(j), products into set j & 1
      const int b = j & 1;
      if (!mbar_wait(&ctl->fb[b], ph_fb[b], abort_flag, wait_cycles)) return false;
      owe_fb[b] = 0;
      ph_fb[b] ^= 1;
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB + b * kLowNS * LB_PLANE);
      const uint32_t dset = tmem_base + b * 256;
      // only the first kLowM of the copy's LBK k are modes; the rest is zero padding
#pragma unroll
      for (int jj = 0; jj < kLowM / 16; ++jj) {
#pragma unroll
        for (int i = 0; i < kLowNS; ++i)
          umma(dset + i * LBN, sdesc(a0 + i * LA_PLANE) + 2 * jj, sdesc(b0) + 2 * jj,
               idesc_f16(BF16, BM, (kLowNS - i) * LBN), (jj > 0 || i > 0) ? 1u : 0u);
      }
      umma_commit(&ctl->md[b]);
      owe_md[b] = 1;
      return true;
    };
    if (threadIdx.x == 0) {
      tmap_acquire(ma);
      tmap_acquire(mb);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&ctl->fa, kLowNS * LA_PLANE);
#pragma unroll
      for (int p = 0; p < kLowNS; ++p) tma_load_2d(sA + p * LA_PLANE, ma, &ctl->fa, 0, p * S.nxp + m0);
      owe_fa = 1;
      issue_b(0);
      bool ok = mbar_wait(&ctl->fa, ph_fa, abort_flag, wait_cycles);
      if (ok) {
        owe_fa = 0;
        ph_fa ^= 1;
        ok = issue_mma(0);
      }
      if (ok && nt > 1) issue_b(1);
    }
    const int m = m0 + row;
    const float sa = pow2f(static_cast<int>(S.low_jt_e[min(m, S.nxp - 1)]) - 16);
    const size_t nn = static_cast<size_t>(S.nx) * S.ny;
    for (int j = 0; j < nt; ++j) {
      const int b = j & 1;
      if (threadIdx.x == 0 && !*abort_flag) {
        // B(j + 1) was copied a step ago; once y-tile j's products are complete its B buffer
        // takes the copy of y-tile j + 2, which lands while this step's sums are merged
        if (mbar_wait(&ctl->md[b], ph_md[b], abort_flag, wait_cycles)) {
          owe_md[b] = 0;
          ph_md[b] ^= 1;
          if (j + 1 < nt && issue_mma(j + 1) && j + 2 < nt) issue_b(j + 2);
        }
      }
      __syncthreads();
      if (*abort_flag) {
        failed = true;
        break;
      }
      tc_fence_after();
      const int n0 = j * LBN + cg * kLowInvCols;  // the warp's columns
      float hi[kLowInvCols], lo[kLowInvCols], scl[kLowInvCols];
#pragma unroll
      for (int c = 0; c < kLowInvCols; ++c) {
        hi[c] = 0.f;
        lo[c] = 0.f;
        scl[c] = sa * pow2f(S.low_qy_e[n0 + c]);
      }
      uint32_t v[kLowNS][kLowInvCols];  // the six order sums, loaded together
#pragma unroll
      for (int d = 0; d < kLowNS; ++d)
        tmem_ld8(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + b * 256 + d * LBN +
                     cg * kLowInvCols, v[d]);
      tmem_wait_ld();
#pragma unroll
      for (int d = 0; d < kLowNS; ++d) {
        const float od = pow2f(-8 * d);
#pragma unroll
        for (int c = 0; c < kLowInvCols; ++c) {
          const float t = __uint_as_float(v[d][c]) * scl[c] * od;
          if (d <= 2) {
            float e;
            two_sum(hi[c], t, hi[c], e);
            lo[c] = __fadd_rn(lo[c], e);
          } else {
            lo[c] = __fadd_rn(lo[c], t);
          }
        }
      }
      tc_fence_before();
      if (m < S.nx) {
#pragma unroll
        for (int c = 0; c < kLowInvCols; ++c) {
          const int y = n0 + c;
          if (y < S.ny) {
            const f2 v = df_norm(hi[c], lo[c]);
            const size_t g = static_cast<size_t>(y) * S.nx + m;
            S.low_z[g] = v.hi;
            S.low_z[nn + g] = v.lo;
          }
        }
      }
      __syncthreads();  // TMEM set b and B buffer b are free for y-tile j + 2
    }
  }
  if (threadIdx.x == 0) {
    // after an abort: copies still in flight land and committed MMAs complete before the CTA
    // frees its TMEM and leaves
    const long long t0 = clock64();
    if (owe_fa) while (!mbar_try(&ctl->fa, ph_fa) && clock64() - t0 < kWaitCycles / 4) {}
    for (int b = 0; b < 2; ++b) {
      if (owe_fb[b]) while (!mbar_try(&ctl->fb[b], ph_fb[b]) && clock64() - t0 < kWaitCycles / 4) {}
      if (owe_md[b]) while (!mbar_try(&ctl->md[b], ph_md[b]) && clock64() - t0 < kWaitCycles / 4) {}
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kLowInvTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0 && ctl->abort_flag) atomicExch(err, 1);
}

// The slices of one double-float value on a single lane (the packed routine on lane x).
template <bool BF16>
__device__ __forceinline__ void slice_codes_df(float vh, float vl, float s, float is,
                                               uint16_t (&code)[kLowNS]) {
  uint32_t c2[kLowNS];
  slice_codes2_df<BF16, kLowNS>(make_float2(vh, 0.f), make_float2(vl, 0.f), make_float2(s, s),
                                make_float2(is, is), c2);
#pragma unroll
  for (int k = 0; k < kLowNS; ++k) code[k] = static_cast<uint16_t>(c2[k] & 0xffffu);
}

// Middle of the low-mode correction, one block per (problem, 128 rows of x) (the inverse
// product's items): G = the forward tiles' shares summed in tile order, G' = w o G, and the
// block's rows of J^T, J^T[x][ky] = sum_kx G'[ky][kx] Qx[x][kx], by compensated dot products of
// double-float operands (Ogita-Rump-Oishi), each row then cut into six slices with its block
// exponent (the inverse product's A operand).  Lane ky reads its row of G' from shared memory;
// the block's rows of Qx_low are staged there transposed, so that a warp takes the values of two
// adjacent rows at one kx by one 8-byte broadcast load, and eight rows run as four packed
// chains.
constexpr int kQsStride = BM + 2;  // [kx][row] stride: even (8-byte pairs), 2-way staging conflicts
template <bool BF16>
__global__ void __launch_bounds__(256)
k_low_mid(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
          const int* __restrict__ n_items, int mode) {
  __shared__ float gh[kLowM][kLowM + 1], gl[kLowM][kLowM + 1];
  __shared__ __align__(16) float qs[2][kLowM][kQsStride];  // Qx_low rows of the block: hi, lo
  const int total = *n_items;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    if (!slot_runs(S.sc, mode) || S.lowm_x == 0) continue;
    const float* qx_h = S.low_qxd;
    const float* qx_l = S.low_qxd + static_cast<size_t>(S.nxp) * kLowM;
    const int xb = it.tile * BM;
    for (int e = t; e < BM * kLowM; e += 256) {
      const int r = e / kLowM, kx = e - r * kLowM;
      const size_t a = static_cast<size_t>(xb + r) * kLowM + kx;
      qs[0][kx][r] = __ldg(qx_h + a);
      qs[1][kx][r] = __ldg(qx_l + a);
    }
    for (int e = t; e < kLowM * kLowM; e += 256) {
      f2 g{0.f, 0.f};
      for (int tt = 0; tt < S.n_l1_tiles; ++tt) {
        const float* gp = S.low_gp + static_cast<size_t>(tt) * 2 * kLowM * kLowM;
        g = df_add(g, f2{gp[e], gp[kLowM * kLowM + e]});
      }
      const int ky = e / kLowM, kx = e - ky * kLowM;
      const float sw = S.lamy[min(ky, S.nyp - 1)] + S.lamx[min(kx, S.nxp - 1)];
      const bool ok = ky < S.lowm_y && kx < S.lowm_x && sw > 0.f;
      g = ok ? df_mul(g, spectral_weight_of(S.wnorm, sw)) : f2{0.f, 0.f};
      gh[ky][kx] = g.hi;
      gl[ky][kx] = g.lo;
    }
    __syncthreads();
    uint16_t* jt = static_cast<uint16_t*>(S.low_jt);
    const size_t plane = static_cast<size_t>(S.nxp) * kLowK3;
    // the warp's 16 rows of the block, eight at a time: four packed pairs of independent chains
    constexpr int kRowsPerGroup = 8;
    for (int rb = warp * (BM / 8); rb < (warp + 1) * (BM / 8); rb += kRowsPerGroup) {
      CompDotDF2 acc[kRowsPerGroup / 2];
#pragma unroll 4
      for (int kx = 0; kx < kLowM; ++kx) {
        const float ah = gh[lane][kx], al = gl[lane][kx];
#pragma unroll
        for (int q = 0; q < kRowsPerGroup / 2; ++q) {
          const float2 bh = *reinterpret_cast<const float2*>(&qs[0][kx][rb + 2 * q]);
          const float2 bl = *reinterpret_cast<const float2*>(&qs[1][kx][rb + 2 * q]);
          acc[q].add(make_float2(ah, ah), make_float2(al, al), bh, bl);
        }
      }
#pragma unroll
      for (int r = 0; r < kRowsPerGroup; ++r) {
        const int x = xb + rb + r;
        const CompDotDF2& d = acc[r / 2];
        const f2 j = (r & 1) ? df_norm(d.s.y, d.c.y) : df_norm(d.s.x, d.c.x);
        const int E = low_block_exp(warp_max(fabsf(j.hi)));
        uint16_t code[kLowNS];
        slice_codes_df<BF16>(j.hi, j.lo, pow2f(8 - E), pow2f(E - 8), code);
#pragma unroll
        for (int p = 0; p < kLowNS; ++p) {
          jt[p * plane + static_cast<size_t>(x) * kLowK3 + lane] = code[p];
          jt[p * plane + static_cast<size_t>(x) * kLowK3 + kLowM + lane] = 0;  // padding columns
        }
        if (lane == 0) S.low_jt_e[x] = static_cast<int8_t>(E);
      }
    }
    __syncthreads();  // gh, gl and qs are rewritten by the next item
  }
}

template <bool BF16, int STAGE>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_prec_tc<BF16, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

template <bool BF16>
void launch_all(const LaunchCfg& c, int stage, int mode, int* err) {
  const long long wc = c.wait_cycles > 0 ? c.wait_cycles : kWaitCycles;
  switch (stage) {
    case 0: k_prec_tc<BF16, 0><<<c.grid, kThreads, SMEM_BYTES, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc); break;
    case 1: k_prec_tc<BF16, 1><<<c.grid, kThreads, SMEM_BYTES, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc); break;
    case 2: k_prec_tc<BF16, 2><<<c.grid, kThreads, SMEM_BYTES, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc); break;
    default: k_prec_tc<BF16, 3><<<c.grid, kThreads, SMEM_BYTES, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc); break;
  }
}

}  // namespace

bool tc_supported() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (p.major != 10 || p.sharedMemPerBlockOptin < static_cast<size_t>(SMEM_BYTES)) return false;
  // one CTA of kThreads threads at kMaxRegs registers each must fit an SM
  int blocks = 0;
  if (set_attr<true, 0>() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_prec_tc<true, 0>, kThreads, SMEM_BYTES) !=
          cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return blocks >= 1;
}

int tc_planes(int) { return NS; }

int tc_block() { return KC; }

template <bool BF16, int KIND>
static cudaError_t set_low_attr() {
  if (KIND == 0)
    return cudaFuncSetAttribute(k_low_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLowSmem);
  return cudaFuncSetAttribute(k_low_inv<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLowInvSmem);
}

cudaError_t tc_init() {
  cudaError_t e = cudaSuccess;
  const cudaError_t r[12] = {set_attr<false, 0>(), set_attr<false, 1>(), set_attr<false, 2>(), set_attr<false, 3>(),
                             set_attr<true, 0>(),  set_attr<true, 1>(),  set_attr<true, 2>(),  set_attr<true, 3>(),
                             set_low_attr<false, 0>(), set_low_attr<false, 1>(), set_low_attr<true, 0>(),
                             set_low_attr<true, 1>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

void launch_low_tc(const LaunchCfg& c, int kind, int mode, int split_kind, int* err) {
  const long long wc = c.wait_cycles > 0 ? c.wait_cycles : kWaitCycles;
  if (split_kind == 0) {
    if (kind == 0) k_low_tc<false><<<c.grid, kLowThreads, kLowSmem, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc);
    else k_low_inv<false><<<c.grid, kLowInvThreads, kLowInvSmem, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc);
  } else {
    if (kind == 0) k_low_tc<true><<<c.grid, kLowThreads, kLowSmem, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc);
    else k_low_inv<true><<<c.grid, kLowInvThreads, kLowInvSmem, c.stream>>>(c.slots, c.items, c.n_items, mode, err, wc);
  }
}

void launch_low_mid(const LaunchCfg& c, int mode, int split_kind) {
  if (split_kind == 0) k_low_mid<false><<<c.grid, 256, 0, c.stream>>>(c.slots, c.items, c.n_items, mode);
  else k_low_mid<true><<<c.grid, 256, 0, c.stream>>>(c.slots, c.items, c.n_items, mode);
}

void launch_tc_fold(const LaunchCfg& c, int mode, int split_kind) {
  if (split_kind == 0) k_tc_fold<false><<<c.grid, 256, 0, c.stream>>>(c.slots, c.tcp, c.items, c.n_items, mode);
  else k_tc_fold<true><<<c.grid, 256, 0, c.stream>>>(c.slots, c.tcp, c.items, c.n_items, mode);
}

void launch_unfold(const LaunchCfg& c, int mode) {
  k_unfold<<<c.grid, 256, 0, c.stream>>>(c.slots, c.tcp, c.items, c.n_items, mode);
}

void launch_prec_tc(const LaunchCfg& c, int stage, int mode, int split_kind, int* err) {
  if (split_kind == 0) launch_all<false>(c, stage, mode, err);
  else launch_all<true>(c, stage, mode, err);
}

void launch_prec_tc_prepare(const LaunchCfg& c, int mode, int split_kind) {
  if (split_kind == 0) k_tc_prepare<false><<<c.grid, 256, 0, c.stream>>>(c.slots, c.items, c.n_items, mode);
  else k_tc_prepare<true><<<c.grid, 256, 0, c.stream>>>(c.slots, c.items, c.n_items, mode);
}

}  // namespace bx
