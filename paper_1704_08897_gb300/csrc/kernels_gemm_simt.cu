// Fast Poisson preconditioner of Sec. 2.2 / Algorithm 1 as four dense transform products on the
// CUDA cores in FP32 arithmetic (the plain path).
//
// z = M Q_y W Q_y^T (M r) Q_x W... written separably on the padded rectangle:
//   stage 0: T1[kx][y]  = sum_x r[y][x]  Qx[x][kx]       (forward transform along x)
//   stage 1: T2[ky][kx] = w(ky,kx) sum_y T1[kx][y] Qy[y][ky]   (along y, times 1/(lam+mu)^2)
//   stage 2: T3[x][ky]  = sum_kx T2[ky][kx] Qx[x][kx]    (inverse along x)
//   stage 3: z[y][x]    = mask(y,x) sum_ky T3[x][ky] Qy[y][ky] (inverse along y), plus partial
//            r.z, z.q per tile (reduced by k_prec_finish)
// Every stage is D[m][n] = sum_k A[m][k] B[n][k] with both operands k-contiguous, written out
// transposed (Out[n][m]) so the next stage again reads a k-contiguous operand.  The division by
// the squared eigenvalue sums is fused into stage 1's epilogue, masking and the CG inner
// products into stage 3's.
//
// Precision.  The weights span (64 / lambda_min)^2, so any rounding noise of the preconditioner
// relative to |r| reappears amplified in the smooth modes of z, and CG pays for it in iterations;
// FP32 products alone cost this operator about 3x the iterations of exact transforms.  Operands
// and stage outputs are therefore double-float (hi, lo) planes, and each product is accumulated
// by the compensated dot product of Ogita, Rump and Oishi (Dot2): TwoProd of the hi parts, a
// TwoSum into the running sum, the error terms and the two hi x lo cross terms into a plain FP32
// compensation.  The result carries about 48 bits.
#include "common.cuh"
#include "kernels.h"

namespace bx {

namespace {

constexpr int BM = 128, BN = 64, BK = 8, NT = 256;

struct StageView {
  const float* A;      // hi plane; the lo plane is A_lo
  const float* A_lo;
  int lda, arows, acols;
  const float* B;      // hi plane; the lo plane follows at B + ldb * ldb
  int ldb;
  float* out;
  float* out_lo;
  int M, N, K;
};

__device__ __forceinline__ StageView stage_view(const SlotDesc& S, int stage) {
  StageView v;
  switch (stage) {
    case 0:
      v = {S.r, S.r_lo, S.nx, S.ny, S.nx, S.qxt, S.nxp, S.t1, S.t1_lo, S.nyp, S.nxp, S.nxp};
      break;
    case 1:
      v = {S.t1, S.t1_lo, S.nyp, S.nxp, S.nyp, S.qyt, S.nyp, S.t2, S.t2_lo, S.nxp, S.nyp, S.nyp};
      break;
    case 2:
      v = {S.t2, S.t2_lo, S.nxp, S.nyp, S.nxp, S.qx, S.nxp, S.t3, S.t3_lo, S.nyp, S.nxp, S.nxp};
      break;
    default:
      v = {S.t3, S.t3_lo, S.nyp, S.nxp, S.nyp, S.qy, S.nyp, nullptr, nullptr, S.nxp, S.nyp, S.nyp};
      break;
  }
  return v;
}

}  // namespace

template <int STAGE>
__global__ void __launch_bounds__(NT)
k_prec_simt(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
            const int* __restrict__ n_items, int mode) {
  __shared__ __align__(16) float As[2][2][BK][BM + 4];  // [buffer][hi, lo][k][m]
  __shared__ __align__(16) float Bs[2][2][BK][BN + 4];
  __shared__ double red[64];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int arow = t >> 1, acol = (t & 1) * 4;  // A tile 128 x 8: 4 per thread and plane
  const int brow = t >> 2, bcol = (t & 3) * 2;  // B tile  64 x 8: 2 per thread and plane
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem item = items[w];
    const SlotDesc& S = slots[item.slot];
    SlotScalars* sc = S.sc;
    const int run = mode == 0 ? sc->active : (mode == 1 ? sc->need_prec : 1);
    if (!run) continue;
    const StageView v = stage_view(S, STAGE);
    const int mtiles = v.M / BM;
    const int m0 = (item.tile % mtiles) * BM;
    const int n0 = (item.tile / mtiles) * BN;
    const float* B_lo = v.B + (size_t)v.ldb * v.ldb;

    float ra[2][4], rb[2][2];
    auto load = [&](int k0) {
      const int am = m0 + arow, ak = k0 + acol;
      if (STAGE == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = am < v.arows && ak + j < v.acols;
          ra[0][j] = in ? v.A[(size_t)am * v.lda + ak + j] : 0.f;
          ra[1][j] = in ? v.A_lo[(size_t)am * v.lda + ak + j] : 0.f;
        }
      } else {
        const float4 a0 = *reinterpret_cast<const float4*>(v.A + (size_t)am * v.lda + ak);
        const float4 a1 = *reinterpret_cast<const float4*>(v.A_lo + (size_t)am * v.lda + ak);
        ra[0][0] = a0.x; ra[0][1] = a0.y; ra[0][2] = a0.z; ra[0][3] = a0.w;
        ra[1][0] = a1.x; ra[1][1] = a1.y; ra[1][2] = a1.z; ra[1][3] = a1.w;
      }
      const size_t bo = (size_t)(n0 + brow) * v.ldb + k0 + bcol;
      const float2 b0 = *reinterpret_cast<const float2*>(v.B + bo);
      const float2 b1 = *reinterpret_cast<const float2*>(B_lo + bo);
      rb[0][0] = b0.x; rb[0][1] = b0.y;
      rb[1][0] = b1.x; rb[1][1] = b1.y;
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int j = 0; j < 4; ++j) As[buf][h][acol + j][arow] = ra[h][j];
#pragma unroll
        for (int j = 0; j < 2; ++j) Bs[buf][h][bcol + j][brow] = rb[h][j];
      }
    };

    // Dot2 accumulators of the thread's 8 x 4 outputs: running sum s and compensation c
    float s[8][4], c[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { s[i][j] = 0.f; c[i][j] = 0.f; }

    const int nk = v.K / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][0][kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][0][kk][64 + ty * 4]);
        const float4 l0 = *reinterpret_cast<const float4*>(&As[buf][1][kk][ty * 4]);
        const float4 l1 = *reinterpret_cast<const float4*>(&As[buf][1][kk][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][0][kk][tx * 4]);
        const float4 bl = *reinterpret_cast<const float4*>(&Bs[buf][1][kk][tx * 4]);
        const float ah[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float al[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
        const float bh[4] = {b0.x, b0.y, b0.z, b0.w};
        const float bo[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float p = __fmul_rn(ah[i], bh[j]);
            const float pe = __fmaf_rn(ah[i], bh[j], -p);
            float e;
            two_sum(s[i][j], p, s[i][j], e);
            c[i][j] = __fadd_rn(c[i][j], __fadd_rn(e, __fmaf_rn(ah[i], bo[j], __fmaf_rn(al[i], bh[j], pe))));
          }
      }
      if (kt + 1 < nk) store(buf ^ 1);
      __syncthreads();
    }

    // epilogue: element (m, n) of D goes to Out[n][m] as a normalised double-float pair
    CompDotDF c_rz, c_zq;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int mb = m0 + h * 64 + ty * 4;
        f2 o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = df_norm(s[h * 4 + i][j], c[h * 4 + i][j]);
        if (STAGE == 1) {
#pragma unroll
          for (int i = 0; i < 4; ++i) o[i] = df_mul(o[i], spectral_weight(S, mb + i, n));
        }
        if (STAGE <= 2) {
          *reinterpret_cast<float4*>(v.out + (size_t)n * v.M + mb) =
              make_float4(o[0].hi, o[1].hi, o[2].hi, o[3].hi);
          *reinterpret_cast<float4*>(v.out_lo + (size_t)n * v.M + mb) =
              make_float4(o[0].lo, o[1].lo, o[2].lo, o[3].lo);
        } else if (S.mir_out) {
          // one mirror class of a folded slot: its result g, unmasked (k_unfold combines the
          // classes, masks and forms the dot products)
          const int y = n;
          if (y < S.ny) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int x = mb + i;
              if (x < S.nx) {
                S.z[y * S.nx + x] = o[i].hi;
                S.z_lo[y * S.nx + x] = o[i].lo;
              }
            }
          }
        } else {
          const int y = n;
          if (y < S.ny) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int x = mb + i;
              if (x < S.nx) {
                const int g = y * S.nx + x;
                const f2 zv = S.mask[g] ? o[i] : f2{0.f, 0.f};
                S.z[g] = zv.hi;
                S.z_lo[g] = zv.lo;
                c_rz.add(S.r[g], S.r_lo[g], zv.hi, zv.lo);
                c_zq.add(zv.hi, zv.lo, S.q[g], S.q_lo[g]);
              }
            }
          }
        }
      }
    }
    if (STAGE == 3 && !S.mir_out) {  // a class problem leaves no partial sums
      double d_rz = c_rz.value(), d_zq = c_zq.value();
      block_sum2<NT>(d_rz, d_zq, red);
      if (t == 0) {  // tile partials; k_prec_finish forms rho and beta from them
        S.part[item.tile * 4 + 2] = d_rz;
        S.part[item.tile * 4 + 3] = d_zq;
      }
    }
    __syncthreads();
  }
}

// The residuals of the mirror classes of a folded slot (CUDA-core path): one thread per class
// node (tiles of 32 x 8), the signed sums of r at the node and its mirrors in double-float (the
// even class adds, the odd class subtracts; a middle node, its own mirror, counts once in the even
// class and not in the odd one), written to each class problem's residual planes.
__global__ void __launch_bounds__(256)
k_simt_fold(const SlotDesc* __restrict__ slots, const SlotDesc* __restrict__ tcp,
            const WorkItem* __restrict__ items, const int* __restrict__ n_items, int mode) {
  const int total = *n_items;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    const int run = mode == 0 ? sc->active : (mode == 1 ? sc->need_prec : 1);
    if (!run) continue;
    const bool fx = (S.mir & 1) != 0, fy = (S.mir & 2) != 0;
    const int ntx = (S.mhx + 31) >> 5;
    const int x = (it.tile % ntx) * 32 + lane, y = (it.tile / ntx) * 8 + warp;
    if (x >= S.mhx || y >= S.mhy) continue;
    const int xx = fx ? S.nx - 1 - x : x, yy = fy ? S.ny - 1 - y : y;
    const bool xmid = xx == x, ymid = yy == y;
    const size_t gy = static_cast<size_t>(y) * S.nx, gyy = static_cast<size_t>(yy) * S.nx;
    const f2 a{S.r[gy + x], S.r_lo[gy + x]};
    const f2 b = xmid ? f2{0.f, 0.f} : f2{S.r[gy + xx], S.r_lo[gy + xx]};
    const f2 c = ymid ? f2{0.f, 0.f} : f2{S.r[gyy + x], S.r_lo[gyy + x]};
    const f2 d = (xmid || ymid) ? f2{0.f, 0.f} : f2{S.r[gyy + xx], S.r_lo[gyy + xx]};
    const f2 e0 = df_add(a, b), o0 = df_add(a, df_neg(b));
    const f2 e1 = df_add(c, d), o1 = df_add(c, df_neg(d));
    f2 v[4] = {df_add(e0, e1), df_add(o0, o1), df_add(e0, df_neg(e1)), df_add(o0, df_neg(o1))};
    if (xmid && fx) v[1] = v[3] = f2{0.f, 0.f};  // the odd x classes vanish at the middle column
    if (ymid && fy) v[2] = v[3] = f2{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (((k & 1) && !fx) || ((k & 2) && !fy)) continue;
      const SlotDesc& T = tcp[kMirClasses * it.slot + k];
      const size_t gi = static_cast<size_t>(y) * T.nx + x;
      T.r[gi] = v[k].hi;
      T.r_lo[gi] = v[k].lo;
    }
  }
}

void launch_simt_fold(const LaunchCfg& c, int mode) {
  k_simt_fold<<<c.grid, 256, 0, c.stream>>>(c.slots, c.tcp, c.items, c.n_items, mode);
}

void launch_prec_simt(const LaunchCfg& c, int stage, int mode) {
  switch (stage) {
    case 0: k_prec_simt<0><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
    case 1: k_prec_simt<1><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
    case 2: k_prec_simt<2><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
    default: k_prec_simt<3><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
  }
}

}  // namespace bx
