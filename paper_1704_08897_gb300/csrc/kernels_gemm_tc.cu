// Fast Poisson preconditioner (Sec. 2.2 / Algorithm 1) on the 5th-generation tensor cores.
//
// The four separable transform products of the preconditioner (see kernels_gemm_simt.cu for the
// stage equations) run as tcgen05 MMAs.  This operator is so ill-conditioned that a plain
// 16-bit operand ruins the preconditioner (rounding noise after the 1/(lam+mu)^2 scaling lands
// in rough modes, and CG stops converging), so every operand is stored as a sum of 16-bit planes:
//   FP16: v = hi + lo            (22 significant bits), products hi*hi + hi*lo + lo*hi
//   BF16: v = hi + mid + lo      (24 significant bits), the six products of order <= 2
// with FP32 accumulation in TMEM.  FP16 planes carry power-of-two scales (data: from the residual
// norm; transform matrices: 2^6) so neither overflow nor underflow occurs; the scales are
// removed exactly in the epilogues.  The tensor core's FP32 accumulation truncates, so its error
// grows with every k-step: each 64-wide k-block is therefore accumulated into a fresh TMEM buffer
// (a ring of four) and the epilogue warps add the k-block sums into a compensated (hi, lo)
// register pair, which keeps the product's error at the level of a 64-term FP32 sum.
//
// Kernel structure (one CTA per SM, persistent over the (slot, tile) work list):
//   warp 0      : TMA producer, 128B-swizzled K-major tiles of every plane into a smem ring
//   warp 1      : TMEM allocation; lane 0 issues the MMAs and the tcgen05.commit arrivals
//   warps 2..5  : k-block sums TMEM -> compensated registers; then the epilogue: next stage's
//                 planes written transposed
//                 (Out[n][m], coalesced along m), with the stage's fused work (eigenvalue
//                 weights; masking, FP64 dot products and the CG scalars in the last stage).
// Every wait on an mbarrier is bounded; on time-out the CTA raises an error flag, drains its
// outstanding copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace bx {
namespace {

constexpr int BM = 128, BN = 64, BK = 64;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at 2 GHz
constexpr int kChunks = 4;                       // TMEM ring of k-block accumulators
constexpr int kTmemCols = kChunks * BN;

template <int NS>
struct TcCfg {
  static constexpr int STAGES = NS == 2 ? 4 : 3;
  static constexpr int A_PLANE = BM * BK * 2;
  static constexpr int B_PLANE = BN * BK * 2;
  static constexpr int STAGE_BYTES = NS * (A_PLANE + B_PLANE);
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 512;
};

struct Ctl {
  uint64_t full[4];
  uint64_t empty[4];
  uint64_t tfull[kChunks];
  uint64_t tempty[kChunks];
  uint64_t drain;
  uint32_t tmem;
  int abort_flag;
  int last;
  int pad;
  double red[8];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false on time-out or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tmap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tmap))
               : "memory");
}

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row core groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;            // leading-dimension offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;    // stride between 8-row groups
  d |= static_cast<uint64_t>(1) << 46;            // descriptor version
  d |= static_cast<uint64_t>(2) << 61;            // 128-byte swizzle
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
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16-bit planes of one value (exact differences: Sterbenz).
template <bool BF16>
__device__ __forceinline__ void split_store(uint16_t* base, size_t plane, size_t idx, float v, int NS) {
  if (BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    base[idx] = __bfloat16_as_ushort(h);
    base[plane + idx] = __bfloat16_as_ushort(m);
    if (NS > 2) base[2 * plane + idx] = __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(m)));
  } else {
    const __half h = __float2half_rn(v);
    base[idx] = __half_as_ushort(h);
    base[plane + idx] = __half_as_ushort(__float2half_rn(v - __half2float(h)));
  }
}

__device__ __forceinline__ bool slot_runs(const SlotScalars* sc, int mode) {
  return mode == 0 ? sc->active != 0 : (mode == 1 ? sc->need_prec != 0 : true);
}

struct TcStage {
  int M, N, K;
  void* out;  // next stage's planes, or nullptr in the last stage
};

__device__ __forceinline__ TcStage tc_stage(const SlotDesc& S, int stage) {
  switch (stage) {
    case 0: return {S.nyp, S.nxp, S.nxp, S.tc_t1};
    case 1: return {S.nxp, S.nyp, S.nyp, S.tc_t2};
    case 2: return {S.nyp, S.nxp, S.nxp, S.tc_t3};
    default: return {S.nxp, S.nyp, S.nyp, nullptr};
  }
}

template <int NS, bool BF16, int STAGE>
__global__ void __launch_bounds__(kThreads, 1)
k_prec_tc(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
          const int* __restrict__ n_items, int mode, int* __restrict__ err) {
  using C = TcCfg<NS>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + C::STAGES * C::STAGE_BYTES);
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = *n_items;
  constexpr uint32_t IDESC = idesc_f16(BF16, BM, BN);
  const float bdescale = BF16 ? 1.f : 1.f / 64.f;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
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
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
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
          if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_flag)) break;
          mbar_expect_tx(&ctl->full[stage], C::STAGE_BYTES);
          unsigned char* sa = smem + stage * C::STAGE_BYTES;
          unsigned char* sb = sa + NS * C::A_PLANE;
#pragma unroll
          for (int p = 0; p < NS; ++p) tma_load_2d(sa + p * C::A_PLANE, ma, &ctl->full[stage], kb * BK, p * v.M + m0);
#pragma unroll
          for (int p = 0; p < NS; ++p) tma_load_2d(sb + p * C::B_PLANE, mb, &ctl->full[stage], kb * BK, p * v.N + n0);
          ++issued;
          if (++stage == C::STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (*abort_flag) {
        // let the copies already issued (at most one per ring slot) land before the CTA leaves
        int s = stage;
        uint32_t ph = phase;
        for (int k = 0; k < C::STAGES && k < issued; ++k) {
          if (s == 0) {
            s = C::STAGES - 1;
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
      int stage = 0;
      uint32_t phase = 0;
      int chunk = 0;  // k-blocks issued so far (position in the TMEM ring)
      bool ok = true;
      for (int w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
        const WorkItem it = items[w];
        const SlotDesc& S = slots[it.slot];
        if (!slot_runs(S.sc, mode)) continue;
        const TcStage v = tc_stage(S, STAGE);
        for (int kb = 0; kb < v.K / BK; ++kb) {
          const int cb = chunk % kChunks;
          if (!mbar_wait(&ctl->tempty[cb], ((chunk / kChunks) & 1) ^ 1, abort_flag) ||
              !mbar_wait(&ctl->full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + cb * BN;
          const uint32_t sa = smem_u32(smem + stage * C::STAGE_BYTES);
          const uint32_t sb = sa + NS * C::A_PLANE;
#pragma unroll
          for (int j = 0; j < BK / 16; ++j) {
            // products of total order <= NS-1 (hi*hi, hi*lo, lo*hi, ...)
#pragma unroll
            for (int pa = 0; pa < NS; ++pa) {
#pragma unroll
              for (int pb = 0; pb + pa < NS; ++pb) {
                const uint64_t ad = sdesc(sa + pa * C::A_PLANE) + 2 * j;
                const uint64_t bd = sdesc(sb + pb * C::B_PLANE) + 2 * j;
                umma(d_tmem, ad, bd, IDESC, (j | pa | pb) != 0 ? 1u : 0u);
              }
            }
          }
          umma_commit(&ctl->empty[stage]);
          umma_commit(&ctl->tfull[cb]);
          if (++stage == C::STAGES) {
            stage = 0;
            phase ^= 1;
          }
          ++chunk;
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
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31 are this warp's
    const int ew = warp - 2;
    const int row = quarter * 32 + lane;
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
      // compensated sum over the k-blocks of this tile
      float hi[BN], lo[BN];
#pragma unroll
      for (int i = 0; i < BN; ++i) {
        hi[i] = 0.f;
        lo[i] = 0.f;
      }
      bool fail_all = false;
      for (int kb = 0; kb < v.K / BK; ++kb) {
        const int cb = chunk % kChunks;
        // all four epilogue warps leave together if any of them gave up waiting
        const uint32_t fail = mbar_wait(&ctl->tfull[cb], (chunk / kChunks) & 1, abort_flag) ? 0u : 1u;
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
#pragma unroll
        for (int c = 0; c < BN / 32; ++c) {
          uint32_t r[32];
          tmem_ld32(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + cb * BN + c * 32, r);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            float e;
            two_sum(hi[c * 32 + i], __uint_as_float(r[i]), hi[c * 32 + i], e);
            lo[c * 32 + i] = __fadd_rn(lo[c * 32 + i], e);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->tempty[cb]);
        ++chunk;
      }
      if (fail_all) break;
      const float inv_scale = (STAGE == 3) ? 1.f / sc->pscale : 1.f;
      const float lamx_m = (STAGE == 1 && m < S.nx) ? S.lamx[m] : 0.f;
      double d_rz = 0.0, d_zq = 0.0;
      const size_t plane = static_cast<size_t>(v.M) * v.N;
#pragma unroll
      for (int i = 0; i < BN; ++i) {
        const int n = n0 + i;
        float val = __fadd_rn(hi[i], lo[i]) * bdescale;
        if (STAGE == 1) {
          float wgt = 0.f;
          if (m < S.nx && n < S.ny) {
            const float s = S.lamy[n] + lamx_m;
            wgt = (s > 0.f) ? S.wnorm / (s * s) : 0.f;
          }
          val *= wgt;
        }
        if (STAGE <= 2) {
          split_store<BF16>(static_cast<uint16_t*>(v.out), plane, static_cast<size_t>(n) * v.M + m, val, NS);
        } else if (n < S.ny && m < S.nx) {
          const int g = n * S.nx + m;
          const float zv = S.mask[g] ? val * inv_scale : 0.f;
          S.z[g] = zv;
          d_rz += (double)S.r[g] * (double)zv;
          d_zq += (double)zv * (double)S.q[g];
        }
      }
      if (STAGE == 3) {
        // tile partials of r.z and z.q, then the slot's last tile forms rho and beta
        d_rz = warp_sum(d_rz);
        d_zq = warp_sum(d_zq);
        if (lane == 0) {
          ctl->red[2 * ew] = d_rz;
          ctl->red[2 * ew + 1] = d_zq;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
        if (ew == 0 && lane == 0) {
          const double a = (ctl->red[0] + ctl->red[2]) + (ctl->red[4] + ctl->red[6]);
          const double b = (ctl->red[1] + ctl->red[3]) + (ctl->red[5] + ctl->red[7]);
          S.part[it.tile * 4 + 0] = a;
          S.part[it.tile * 4 + 1] = b;
          __threadfence();
          const unsigned prev = atomicAdd(&sc->cnt[4], 1u);
          const int last = (prev == static_cast<unsigned>(S.n_tc_tiles) - 1) ? 1 : 0;
          if (last) {
            __threadfence();
            sc->cnt[4] = 0u;
          }
          ctl->last = last;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
        if (ctl->last) {
          double a = 0.0, b = 0.0;
          const int t = ew * 32 + lane;
          for (int k = t; k < S.n_tc_tiles; k += 32 * kEpiWarps) {
            a += __ldcg(&S.part[k * 4 + 0]);
            b += __ldcg(&S.part[k * 4 + 1]);
          }
          a = warp_sum(a);
          b = warp_sum(b);
          asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
          if (lane == 0) {
            ctl->red[2 * ew] = a;
            ctl->red[2 * ew + 1] = b;
          }
          asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
          if (ew == 0 && lane == 0) {
            const double rz = (ctl->red[0] + ctl->red[2]) + (ctl->red[4] + ctl->red[6]);
            const double zq = (ctl->red[1] + ctl->red[3]) + (ctl->red[5] + ctl->red[7]);
            finish_preconditioner(S, rz, zq, mode);
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
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

// Residual -> scaled 16-bit planes of the first stage's A operand (padding stays zero).
template <int NS, bool BF16>
__global__ void __launch_bounds__(kVecThreads)
k_tc_prepare(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
             const int* __restrict__ n_items, int mode) {
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    if (!slot_runs(sc, mode)) continue;
    // FP16: scale so that ||r||_2 is about 2^12; every transform stage keeps |values| <= ||r||_2
    float s = 1.f;
    if (!BF16 && mode != 2 && sc->rr > 0.0) {
      int e;
      frexp(sqrt(sc->rr), &e);
      s = ldexpf(1.f, 12 - e);
    }
    if (it.tile == 0 && threadIdx.x == 0) sc->pscale = s;
    const int n = S.nx * S.ny;
    const int e0 = it.tile * kVecChunk;
    const int e1 = min(n, e0 + kVecChunk);
    const size_t plane = static_cast<size_t>(S.nyp) * S.nxp;
    uint16_t* out = static_cast<uint16_t*>(S.tc_r);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int y = e / S.nx, x = e - y * S.nx;
      split_store<BF16>(out, plane, static_cast<size_t>(y) * S.nxp + x, S.r[e] * s, NS);
    }
  }
}

template <int NS, bool BF16, int STAGE>
void launch_stage(const LaunchCfg& c, int mode, int* err) {
  using C = TcCfg<NS>;
  k_prec_tc<NS, BF16, STAGE><<<c.grid, kThreads, C::SMEM, c.stream>>>(c.slots, c.items, c.n_items, mode, err);
}

template <int NS, bool BF16, int STAGE>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_prec_tc<NS, BF16, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcCfg<NS>::SMEM);
}

template <int NS, bool BF16>
void launch_all(const LaunchCfg& c, int stage, int mode, int* err) {
  switch (stage) {
    case 0: launch_stage<NS, BF16, 0>(c, mode, err); break;
    case 1: launch_stage<NS, BF16, 1>(c, mode, err); break;
    case 2: launch_stage<NS, BF16, 2>(c, mode, err); break;
    default: launch_stage<NS, BF16, 3>(c, mode, err); break;
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
  return p.major == 10 && p.sharedMemPerBlockOptin >= static_cast<size_t>(TcCfg<3>::SMEM);
}

int tc_planes(int split_kind) { return split_kind == 0 ? 2 : 3; }

cudaError_t tc_init() {
  cudaError_t e = cudaSuccess;
  cudaError_t r[8] = {set_attr<2, false, 0>(), set_attr<2, false, 1>(), set_attr<2, false, 2>(),
                      set_attr<2, false, 3>(), set_attr<3, true, 0>(),  set_attr<3, true, 1>(),
                      set_attr<3, true, 2>(),  set_attr<3, true, 3>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

void launch_prec_tc(const LaunchCfg& c, int stage, int mode, int split_kind, int* err) {
  if (split_kind == 0) launch_all<2, false>(c, stage, mode, err);
  else launch_all<3, true>(c, stage, mode, err);
}

void launch_prec_tc_prepare(const LaunchCfg& c, int mode, int split_kind) {
  if (split_kind == 0) k_tc_prepare<2, false><<<c.grid, kVecThreads, 0, c.stream>>>(c.slots, c.items, c.n_items, mode);
  else k_tc_prepare<3, true><<<c.grid, kVecThreads, 0, c.stream>>>(c.slots, c.items, c.n_items, mode);
}

}  // namespace bx
