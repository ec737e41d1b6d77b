// Fast Poisson preconditioner of Sec. 2.2 / Algorithm 1 as four dense transform products, FP32
// on the CUDA cores (the plain path).
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
#include "common.cuh"
#include "kernels.h"

namespace bx {

namespace {

constexpr int BM = 128, BN = 64, BK = 16, NT = 256;

struct StageView {
  const float* A;
  int lda, arows, acols;
  const float* B;
  int ldb;
  float* out;
  int M, N, K;
};

__device__ __forceinline__ StageView stage_view(const SlotDesc& S, int stage) {
  StageView v;
  switch (stage) {
    case 0:
      v = {S.r, S.nx, S.ny, S.nx, S.qxt, S.nxp, S.t1, S.nyp, S.nxp, S.nxp};
      break;
    case 1:
      v = {S.t1, S.nyp, S.nxp, S.nyp, S.qyt, S.nyp, S.t2, S.nxp, S.nyp, S.nyp};
      break;
    case 2:
      v = {S.t2, S.nxp, S.nyp, S.nxp, S.qx, S.nxp, S.t3, S.nyp, S.nxp, S.nxp};
      break;
    default:
      v = {S.t3, S.nyp, S.nxp, S.nyp, S.qy, S.nyp, nullptr, S.nxp, S.nyp, S.nyp};
      break;
  }
  return v;
}

}  // namespace

template <int STAGE>
__global__ void __launch_bounds__(NT)
k_prec_simt(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
            const int* __restrict__ n_items, int mode) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  __shared__ double red[64];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int arow = t >> 1, acol = (t & 1) * 8;  // A tile 128 x 16: 8 per thread
  const int brow = t >> 2, bcol = (t & 3) * 4;  // B tile  64 x 16: 4 per thread
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

    float ra[8], rb[4];
    auto load = [&](int k0) {
      const int am = m0 + arow, ak = k0 + acol;
      if (STAGE == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          ra[j] = (am < v.arows && ak + j < v.acols) ? v.A[(size_t)am * v.lda + ak + j] : 0.f;
      } else {
        const float4* pa = reinterpret_cast<const float4*>(v.A + (size_t)am * v.lda + ak);
        const float4 a0 = pa[0], a1 = pa[1];
        ra[0] = a0.x; ra[1] = a0.y; ra[2] = a0.z; ra[3] = a0.w;
        ra[4] = a1.x; ra[5] = a1.y; ra[6] = a1.z; ra[7] = a1.w;
      }
      const float4 b0 = *reinterpret_cast<const float4*>(v.B + (size_t)(n0 + brow) * v.ldb + k0 + bcol);
      rb[0] = b0.x; rb[1] = b0.y; rb[2] = b0.z; rb[3] = b0.w;
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int j = 0; j < 8; ++j) As[buf][acol + j][arow] = ra[j];
#pragma unroll
      for (int j = 0; j < 4; ++j) Bs[buf][bcol + j][brow] = rb[j];
    };

    // Each 16-term chunk of the k sum is accumulated in FP32 (c); chunks are merged into the
    // (hi, lo) pair with an error-free TwoSum, so the sum's error does not grow with K.
    float c[8][4], hi[8][4], lo[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { c[i][j] = 0.f; hi[i][j] = 0.f; lo[i][j] = 0.f; }

    const int nk = v.K / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) c[i][j] = fmaf(a[i], b[j], c[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float e;
          two_sum(hi[i][j], c[i][j], hi[i][j], e);
          lo[i][j] = __fadd_rn(lo[i][j], e);
          c[i][j] = 0.f;
        }
      if (kt + 1 < nk) store(buf ^ 1);
      __syncthreads();
    }

    // epilogue: element (m, n) of D goes to Out[n][m]
    CompDot c_rz, c_zq;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int mb = m0 + h * 64 + ty * 4;
        float o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = __fadd_rn(hi[h * 4 + i][j], lo[h * 4 + i][j]);
        if (STAGE == 1) {
#pragma unroll
          for (int i = 0; i < 4; ++i) o[i] *= spectral_weight(S, mb + i, n);
        }
        if (STAGE <= 2) {
          *reinterpret_cast<float4*>(v.out + (size_t)n * v.M + mb) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
          const int y = n;
          if (y < S.ny) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int x = mb + i;
              if (x < S.nx) {
                const int g = y * S.nx + x;
                const float zv = S.mask[g] ? o[i] : 0.f;
                S.z[g] = zv;
                c_rz.add(S.r[g], zv);
                c_zq.add(zv, S.q[g]);
              }
            }
          }
        }
      }
    }
    if (STAGE == 3) {
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

void launch_prec_simt(const LaunchCfg& c, int stage, int mode) {
  switch (stage) {
    case 0: k_prec_simt<0><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
    case 1: k_prec_simt<1><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
    case 2: k_prec_simt<2><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
    default: k_prec_simt<3><<<c.grid, NT, 0, c.stream>>>(c.slots, c.items, c.n_items, mode); break;
  }
}

}  // namespace bx
