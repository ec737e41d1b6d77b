// Grid kernels of the PCG extension solve: right-hand side, masked biharmonic apply, CG vector
// update, residual replacement and output.  All are persistent launches over a work list of
// (slot, tile) items so that one launch serves a single solve, a batch or the serving loop.
//
// The operator is eq. (discrete_biharmonic) of Sec. 2.1 with the boundary rules of Algorithm 1
// (Dirichlet padding), half-sample reflection (symmetric) or wrap-around (periodic), evaluated
// matrix-free ("no need to form the 13-banded matrix", Sec. 2.2).
//
// CG vectors are double-float pairs of FP32 planes (hi, lo); see SlotDesc.
#include "async.cuh"
#include "common.cuh"
#include "kernels.h"

namespace bx {

constexpr int kHX = kStTileX + 4;  // 68
constexpr int kHY = kStTileY + 4;  // 36
constexpr int kHalo = kHX * kHY;

__device__ __forceinline__ void tile_origin(const SlotDesc& S, int tile, int& x0, int& y0) {
  const int tx = (S.nx + kStTileX - 1) / kStTileX;
  x0 = (tile % tx) * kStTileX;
  y0 = (tile / tx) * kStTileY;
}

// Map halo position i of the tile to (global index, sign); sign 0 = outside / zero node.
__device__ __forceinline__ int halo_src(const SlotDesc& S, int x0, int y0, int i, float& s) {
  const int ly = i / kHX, lx = i - ly * kHX;
  const int gy = y0 - 2 + ly, gx = x0 - 2 + lx;
  if (gx > S.nx + 1 || gy > S.ny + 1) { s = 0.f; return 0; }
  float sx, sy;
  const int mx = ghost(gx, S.nx, S.bcx, sx);
  const int my = ghost(gy, S.ny, S.bcy, sy);
  s = sx * sy;
  return my * S.nx + mx;
}

// 13-point masked biharmonic of a smem tile (row stride RS) at local (ly+2, lx+2), as a
// compensated FP32 sum (s, c): s + c carries the exact sum of the 13 terms to about 48 bits.
template <bool ANISO, int RS = kHX>
__device__ __forceinline__ CompSum stencil13_acc(const SlotDesc& S, const float* t, int ly, int lx) {
  const float* c = t + (ly + 2) * RS + (lx + 2);
  const float C = c[0];
  const float E0 = c[-1], E1 = c[1], N0 = c[-RS], N1 = c[RS];
  const float D0 = c[-RS - 1], D1 = c[-RS + 1], D2 = c[RS - 1], D3 = c[RS + 1];
  const float F0 = c[-2], F1 = c[2], G0 = c[-2 * RS], G1 = c[2 * RS];
  CompSum acc;
  if (!ANISO) {
    // 20 C - 8 (edges) + 2 (diagonals) + (distance 2); every term is an exact FP32 value
    acc.add(16.f * C);
    acc.add(4.f * C);
    acc.add(-8.f * E0); acc.add(-8.f * E1); acc.add(-8.f * N0); acc.add(-8.f * N1);
    acc.add(2.f * D0); acc.add(2.f * D1); acc.add(2.f * D2); acc.add(2.f * D3);
    acc.add(F0); acc.add(F1); acc.add(G0); acc.add(G1);
  } else {
    acc.add_prod(S.wc, C);
    acc.add_prod(S.wex, E0); acc.add_prod(S.wex, E1);
    acc.add_prod(S.wey, N0); acc.add_prod(S.wey, N1);
    acc.add_prod(S.wd, D0); acc.add_prod(S.wd, D1); acc.add_prod(S.wd, D2); acc.add_prod(S.wd, D3);
    acc.add_prod(S.wfx, F0); acc.add_prod(S.wfx, F1);
    acc.add_prod(S.wfy, G0); acc.add_prod(S.wfy, G1);
    // low parts of the weights: products far below the result's ulp, plain FP32 suffices
    float lo = S.wc_l * C + S.wex_l * (E0 + E1) + S.wey_l * (N0 + N1) +
               S.wd_l * ((D0 + D1) + (D2 + D3)) + S.wfx_l * (F0 + F1) + S.wfy_l * (G0 + G1);
    acc.c = __fadd_rn(acc.c, lo);
  }
  return acc;
}

// The same stencil applied in plain FP32 (for the lo plane of a double-float vector, whose
// contribution is 2^-24 of the hi plane's: its own rounding is far below the result's ulp).
template <bool ANISO, int RS>
__device__ __forceinline__ float stencil13_plain(const SlotDesc& S, const float* t, int ly, int lx) {
  const float* c = t + (ly + 2) * RS + (lx + 2);
  const float e = (c[-1] + c[1]), n = (c[-RS] + c[RS]);
  const float d = (c[-RS - 1] + c[-RS + 1]) + (c[RS - 1] + c[RS + 1]);
  const float f = c[-2] + c[2], g = c[-2 * RS] + c[2 * RS];
  if (!ANISO) return 20.f * c[0] - 8.f * (e + n) + 2.f * d + (f + g);
  return S.wc * c[0] + S.wex * e + S.wey * n + S.wd * d + S.wfx * f + S.wfy * g;
}

template <bool ANISO, int RS = kHX>
__device__ __forceinline__ float stencil13(const SlotDesc& S, const float* t, int ly, int lx) {
  return stencil13_acc<ANISO, RS>(S, t, ly, lx).result();
}

// The isotropic 13-point stencil at two adjacent nodes (x, x+1) of a smem tile with an even row
// stride RS; c points at node x, an even index.  Eleven aligned 8-byte loads cover both
// neighbourhoods, and each lane runs the scalar stencil13_acc's operations in the same order
// (bit-identical results).
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
template <int RS>
__device__ __forceinline__ CompSum2 stencil13_pair_acc(const float* c) {
  static_assert(RS % 2 == 0, "pairs of nodes start on 8-byte boundaries");
  const float2 Cm = ld2(c - 2), C = ld2(c), Cp = ld2(c + 2);                  // row y
  const float2 Nm = ld2(c - RS - 2), N = ld2(c - RS), Np = ld2(c - RS + 2);   // row y-1
  const float2 Sm = ld2(c + RS - 2), Sv = ld2(c + RS), Sp = ld2(c + RS + 2);  // row y+1
  const float2 NN = ld2(c - 2 * RS), SS = ld2(c + 2 * RS);                    // rows y-2, y+2
  const float2 E0 = make_float2(Cm.y, C.x), E1 = make_float2(C.y, Cp.x);
  const float2 D0 = make_float2(Nm.y, N.x), D1 = make_float2(N.y, Np.x);
  const float2 D2 = make_float2(Sm.y, Sv.x), D3 = make_float2(Sv.y, Sp.x);
  CompSum2 acc;
  acc.add(mul2(16.f, C));
  acc.add(mul2(4.f, C));
  acc.add(mul2(-8.f, E0)); acc.add(mul2(-8.f, E1)); acc.add(mul2(-8.f, N)); acc.add(mul2(-8.f, Sv));
  acc.add(mul2(2.f, D0)); acc.add(mul2(2.f, D1)); acc.add(mul2(2.f, D2)); acc.add(mul2(2.f, D3));
  acc.add(Cm); acc.add(Cp); acc.add(NN); acc.add(SS);
  return acc;
}
// plain FP32 stencil of the lo plane at two adjacent nodes
template <int RS>
__device__ __forceinline__ float2 stencil13_pair_plain(const float* c) {
  const float2 Cm = ld2(c - 2), C = ld2(c), Cp = ld2(c + 2);
  const float2 Nm = ld2(c - RS - 2), N = ld2(c - RS), Np = ld2(c - RS + 2);
  const float2 Sm = ld2(c + RS - 2), Sv = ld2(c + RS), Sp = ld2(c + RS + 2);
  const float2 NN = ld2(c - 2 * RS), SS = ld2(c + 2 * RS);
  const float2 E = add2(make_float2(Cm.y, C.x), make_float2(C.y, Cp.x));
  const float2 D = add2(add2(make_float2(Nm.y, N.x), make_float2(N.y, Np.x)),
                        add2(make_float2(Sm.y, Sv.x), make_float2(Sv.y, Sp.x)));
  const float2 F = add2(add2(Cm, Cp), add2(NN, SS));
  float2 v = mul2(20.f, C);
  v = fma2(make_float2(-8.f, -8.f), add2(E, add2(N, Sv)), v);
  v = fma2(make_float2(2.f, 2.f), D, v);
  return add2(v, F);
}

__device__ __forceinline__ double stencil13_f64(const SlotDesc& S, const double* t, int ly, int lx) {
  const double* c = t + (ly + 2) * kHX + (lx + 2);
  return S.dwc * c[0] + S.dwex * (c[-1] + c[1]) + S.dwey * (c[-kHX] + c[kHX]) +
         S.dwd * ((c[-kHX - 1] + c[-kHX + 1]) + (c[kHX - 1] + c[kHX + 1])) +
         S.dwfx * (c[-2] + c[2]) + S.dwfy * (c[-2 * kHX] + c[2 * kHX]);
}

// ---------------------------------------------------------------------------------------------
// Setup: known mask from sign(phi) (Sec. 2.1), b = -M L^2 E_K f in FP64 (Algorithm 1, first
// statement), zero CG state.  Partials: ||b||^2, number of known nodes, number of invalid inputs
// (NaN phi, or a non-finite f at a known node).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kStThreads)
k_setup(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
        const int* __restrict__ n_items, const float* const* __restrict__ phis,
        const float* const* __restrict__ fs, const int* __restrict__ dirs) {
  __shared__ double sf[kHalo];
  __shared__ double red[64];
  __shared__ int s_last;
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    const float* phi = phis[it.slot];
    const float* f = fs[it.slot];
    const bool out_dir = dirs[it.slot] == 0;
    int x0, y0;
    tile_origin(S, it.tile, x0, y0);
    for (int i = threadIdx.x; i < kHalo; i += blockDim.x) {
      float s;
      const int g = halo_src(S, x0, y0, i, s);
      double v = 0.0;
      if (s != 0.f) {
        const float ph = phi[g];
        const bool known = out_dir ? (ph < 0.f) : (ph > 0.f);
        v = known ? (double)s * (double)f[g] : 0.0;
      }
      sf[i] = v;
    }
    __syncthreads();
    double bb = 0.0, cnt = 0.0, bad = 0.0;
    for (int k = threadIdx.x; k < kStTileX * kStTileY; k += blockDim.x) {
      const int ly = k / kStTileX, lx = k - ly * kStTileX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx >= S.nx || gy >= S.ny) continue;
      const int g = gy * S.nx + gx;
      const float ph = phi[g];
      const bool known = out_dir ? (ph < 0.f) : (ph > 0.f);
      if (ph != ph || (known && !isfinite(f[g]))) bad += 1.0;
      double bv = 0.0;
      if (!known) bv = -stencil13_f64(S, sf, ly, lx);
      S.mask[g] = known ? 0 : 1;
      S.b[g] = bv;
      S.xhi[g] = 0.f;
      S.xlo[g] = 0.f;
      S.r[g] = 0.f;
      S.r_lo[g] = 0.f;
      S.p[0][g] = 0.f;
      S.p[1][g] = 0.f;
      S.p_lo[0][g] = 0.f;
      S.p_lo[1][g] = 0.f;
      S.q[g] = 0.f;
      S.q_lo[g] = 0.f;
      S.z[g] = 0.f;
      S.z_lo[g] = 0.f;
      bb += bv * bv;
      cnt += known ? 1.0 : 0.0;
    }
    block_sum2<kStThreads>(bb, cnt, red);
    double nn = bad, dummy = 0.0;
    block_sum2<kStThreads>(nn, dummy, red);
    if (threadIdx.x == 0) {
      S.part[it.tile * 4 + 0] = bb;
      S.part[it.tile * 4 + 1] = cnt;
      S.part[it.tile * 4 + 2] = nn;
    }
    if (last_item_block(&S.sc->cnt[0], S.n_st_tiles, &s_last)) {
      double sums[3];
      reduce_partials<kStThreads, 3>(S.part, S.n_st_tiles, sums, red);
      if (threadIdx.x == 0) {
        const double sb = sums[0], sk = sums[1], sn = sums[2];
        SlotScalars* sc = S.sc;
        // The extension is linear in f: the iteration runs on 2^e b with e chosen so that the
        // root mean square of 2^e b over the unknowns is near 1, which keeps the FP32 vectors
        // and their pairwise products inside FP32's range for any magnitude of f.  A power of
        // two changes no rounding; k_output scales the answer back.
        int e = 0;
        const double n_unk = (double)S.nx * (double)S.ny - sk;
        if (sb > 0.0 && isfinite(sb) && n_unk > 0.0) {
          int k;
          frexp(sb / n_unk, &k);
          e = max(-1000, min(1000, -(k / 2)));
        }
        sc->bexp = e;
        const double sbs = ldexp(sb, 2 * e);
        sc->bb = sbs;
        sc->rr = sbs;
        sc->rr_true = sbs;
        sc->rr_ref = sbs;
        sc->rho = 0.0;
        sc->beta = 0.0;
        sc->alpha = 0.0;
        sc->it = 0;
        sc->fold = 0;
        sc->n_known = (int)sk;
        if (sn > 0.0 || !isfinite(sb)) {
          sc->status = -1;  // EXT_EINVAL: NaN in phi or a non-finite known value
          sc->active = 0;
          sc->need_prec = 0;
        } else if (sb == 0.0) {
          sc->status = ST_OK;  // b = 0: x = 0 is exact
          sc->active = 0;
          sc->need_prec = 0;
        } else {
          sc->status = ST_RUNNING;
          sc->active = 1;
          sc->need_prec = 1;
        }
      }
    }
    __syncthreads();
  }
}

// Set-up, second pass: r = 2^e b as a double-float pair, once the slot's scale exponent e is
// known.
__global__ void __launch_bounds__(kStThreads)
k_rhs_scale(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
            const int* __restrict__ n_items) {
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    if (S.sc->status != ST_RUNNING) continue;
    const int e = S.sc->bexp;
    int x0, y0;
    tile_origin(S, it.tile, x0, y0);
    for (int k = threadIdx.x; k < kStTileX * kStTileY; k += blockDim.x) {
      const int ly = k / kStTileX, lx = k - ly * kStTileX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx >= S.nx || gy >= S.ny) continue;
      const int g = gy * S.nx + gx;
      const f2 v = df_of(ldexp(S.b[g], e));
      S.r[g] = v.hi;
      S.r_lo[g] = v.lo;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Iteration, stage 1: p = z + beta p_old (formed in shared memory including the halo, in
// double-float), q = M L^2 p (Algorithm 1, matvec, with the mask in the epilogue), and p.q as
// partial sums over fixed 64 x 16 node blocks; k_pq_finish then forms alpha = rho / p.q.
//
// q is the double-float pair of the exact 13-point sum of p's hi plane (compensated FP32) plus
// the same stencil of p's lo plane in plain FP32.
//
// Tiles are 64 nodes wide and TY rows high (TY = 16 or 32, chosen per workspace by the
// autotuner).  Each block walks its share of the (slot, tile) list with two shared-memory window
// sets.  For a slot whose rows span a multiple of 16 bytes in the mask (nx % 16 == 0), the window
// set of the block's next tile arrives by tensor copies while it computes the current one: the hi
// and lo planes of z and p_old over rows y0-2 .. y0+TY+1 and columns x0-4 .. x0+67 (two columns
// wider on the left than the halo, so that each copy starts on a 16-byte boundary) and the tile's
// mask bytes.  Cells outside the grid arrive as zeros; the ghost cells of a boundary tile
// (reflected, wrapped or negated copies of grid nodes under the boundary rule) are gathered by
// plain loads.  Tiles of other slots fill the free window set with plain loads.
//
// The p.q partials do not depend on TY: they are per 64 x 16 block (a tile holds TY / 16 of
// them), each thread adds its nodes of a block in step order (the steps cover the block's rows
// in the same order for either TY), the warp adds its lanes in a fixed butterfly and one thread
// the eight warps in order; k_pq_finish adds the blocks in index order, so every tile height
// gives the same bits.
// ---------------------------------------------------------------------------------------------
constexpr int kWX = kStWinX;  // 72: window row, floats
static_assert(kStWinX == kStTileX + 8, "window columns");

template <int TY>
struct StGeom {
  static constexpr int kHYt = TY + 4;                       // halo rows
  static constexpr int kHalo = kHX * kHYt;                   // halo cells
  static constexpr int kWinBytes = kWX * kHYt * 4;           // one FP32 plane window
  static constexpr int kMaskBytes = kStTileX * TY;           // the tile's mask
  static constexpr int kBufBytes = 4 * kWinBytes + kMaskBytes;  // z, z_lo, p, p_lo, mask
  static constexpr int kGhostSlots = 4 * kHYt + 4 * kHX;     // candidate ghost cells of one halo
  static constexpr int kBlocksPerSm = TY == 32 ? 2 : 3;
  static constexpr int kSmemBytes = 2 * kBufBytes + 128;     // two window sets, alignment slack
  static constexpr int kOwn = kStTileX * TY / kStThreads;    // nodes per thread
  static_assert(kWinBytes % 128 == 0 && kBufBytes % 128 == 0, "tensor copy destinations");
  static_assert(kGhostSlots <= 2 * kStThreads, "two ghost candidates per thread");
  static_assert(kOwn * kStThreads == kStTileX * TY && kOwn % 2 == 0, "tile / block size");
  static_assert(kBlocksPerSm * (kSmemBytes + 1024) <= 228 * 1024, "window sets per SM");
};

__device__ __forceinline__ void tile_origin_ty(const SlotDesc& S, int tile, int ty, int& x0, int& y0) {
  const int tx = (S.nx + kStTileX - 1) / kStTileX;
  x0 = (tile % tx) * kStTileX;
  y0 = (tile / tx) * ty;
}

// Candidate k of a tile's ghost cells: the four ghost columns (x = -2, -1, nx, nx+1) over the
// halo's rows, then the four ghost rows over the halo's in-grid columns.  Returns false when the
// candidate lies outside the halo or beyond the second ghost line; (wy, wx) is its window cell.
template <int TY>
__device__ __forceinline__ bool ghost_cell(const SlotDesc& S, int x0, int y0, int k, int& wy,
                                           int& wx) {
  constexpr int kHYt = StGeom<TY>::kHYt;
  if (k < 4 * kHYt) {
    const int j = k / kHYt;
    wy = k - j * kHYt;
    const int gx = j < 2 ? j - 2 : S.nx + (j - 2);
    const int lx = gx - (x0 - 2);
    wx = lx + 2;
    return lx >= 0 && lx < kHX && y0 - 2 + wy <= S.ny + 1;
  }
  const int kk = k - 4 * kHYt;
  const int j = kk / kHX, lx = kk - j * kHX;
  const int gy = j < 2 ? j - 2 : S.ny + (j - 2);
  const int gx = x0 - 2 + lx;
  wy = gy - (y0 - 2);
  wx = lx + 2;
  return wy >= 0 && wy < kHYt && gx >= 0 && gx < S.nx;
}

// Halo cell i of a TY-row tile: (global index, sign); sign 0 = outside / zero node.
template <int TY>
__device__ __forceinline__ int halo_src_ty(const SlotDesc& S, int x0, int y0, int i, float& s) {
  const int ly = i / kHX, lx = i - ly * kHX;
  const int gy = y0 - 2 + ly, gx = x0 - 2 + lx;
  if (gx > S.nx + 1 || gy > S.ny + 1) { s = 0.f; return 0; }
  float sx, sy;
  const int mx = ghost(gx, S.nx, S.bcx, sx);
  const int my = ghost(gy, S.ny, S.bcy, sy);
  s = sx * sy;
  return my * S.nx + mx;
}

// Thread 0: start the tensor copies of the block's next copied tile (the next item at or after
// w_issue whose slot iterates and has stencil maps) into window set n_issued % 2.
template <int TY>
__device__ __forceinline__ void stencil_issue_next(const SlotDesc* __restrict__ slots,
                                                   const WorkItem* __restrict__ items, int total,
                                                   unsigned char* sbuf, uint64_t* full,
                                                   int& w_issue, int& n_issued) {
  using G = StGeom<TY>;
  while (w_issue < total) {
    const WorkItem it = items[w_issue];
    w_issue += gridDim.x;
    const SlotDesc& S = slots[it.slot];
    if (S.st_maps == nullptr || !S.sc->active) continue;
    int x0, y0;
    tile_origin_ty(S, it.tile, TY, x0, y0);
    const unsigned char* maps = static_cast<const unsigned char*>(S.st_maps);
    const int par = S.sc->it & 1;
    const void* src[5] = {maps, maps + 128, maps + 128 * (2 + 2 * par), maps + 128 * (3 + 2 * par),
                          maps + 128 * 6};
#pragma unroll
    for (int k = 0; k < 5; ++k) tmap_acquire(src[k]);
    const int b = n_issued & 1;
    unsigned char* dst = sbuf + b * G::kBufBytes;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&full[b], G::kBufBytes);
#pragma unroll
    for (int k = 0; k < 4; ++k) tma_load_2d(dst + k * G::kWinBytes, src[k], &full[b], x0 - 4, y0 - 2);
    tma_load_2d(dst + 4 * G::kWinBytes, src[4], &full[b], x0, y0);
    ++n_issued;
    return;
  }
}

// Compensated sum of (s, c) pairs over the lanes of groups of W consecutive lanes (W = 16 or 32),
// in a fixed butterfly; the group's total (as FP64) is valid in every lane of the group.
template <int W>
__device__ __forceinline__ double group_sum_comp(float s, float c) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    float e;
    two_sum(s, s2, s, e);
    c = __fadd_rn(c, __fadd_rn(c2, e));
  }
  return (double)s + (double)c;
}

template <bool ANISO, int TY>
__global__ void __launch_bounds__(kStThreads, StGeom<TY>::kBlocksPerSm)
k_stencil(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
          const int* __restrict__ n_items, int* __restrict__ err, long long wait_cycles) {
  using G = StGeom<TY>;
  extern __shared__ unsigned char st_smem_raw[];
  unsigned char* sbuf = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(st_smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  __shared__ __align__(8) uint64_t full[2];
  __shared__ int s_abort;
  __shared__ double blk_sm[TY / 16][kStThreads / 32];  // p.q of each warp in each 16-row block
  const int total = *n_items;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  volatile int* abort_flag = &s_abort;
  int w_issue = blockIdx.x, n_issued = 0;  // thread 0: the tensor-copy cursor
  int n_used = 0;                          // copied windows consumed (uniform over the block)
  if (threadIdx.x == 0) stencil_issue_next<TY>(slots, items, total, sbuf, full, w_issue, n_issued);
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    if (!sc->active) continue;
    const f2 beta = df_of(sc->beta);
    const int par = sc->it & 1;
    const float* __restrict__ pold = S.p[par];
    const float* __restrict__ pold_lo = S.p_lo[par];
    float* __restrict__ pnew = S.p[par ^ 1];
    float* __restrict__ pnew_lo = S.p_lo[par ^ 1];
    const float* __restrict__ z = S.z;
    const float* __restrict__ z_lo = S.z_lo;
    int x0, y0;
    tile_origin_ty(S, it.tile, TY, x0, y0);
    // a tile whose halo lies inside the grid has no ghost cell
    const bool interior = x0 >= 2 && y0 >= 2 && x0 + kStTileX + 2 <= S.nx && y0 + TY + 2 <= S.ny;
    unsigned char* buf;
    if (S.st_maps != nullptr) {
      const int b = n_used & 1;
      buf = sbuf + b * G::kBufBytes;
      // the other window set finished with the previous tile: start the next tile's copies
      if (threadIdx.x == 0 && n_issued == n_used + 1)
        stencil_issue_next<TY>(slots, items, total, sbuf, full, w_issue, n_issued);
      // ghost cells by plain loads, issued before the wait so that both latencies overlap
      int gcell[2] = {-1, -1};
      float gs[2] = {0.f, 0.f};
      f2 gz[2] = {{0.f, 0.f}, {0.f, 0.f}}, gp[2] = {{0.f, 0.f}, {0.f, 0.f}};
      if (!interior) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = threadIdx.x + h * kStThreads;
          int wy, wx;
          if (k < G::kGhostSlots && ghost_cell<TY>(S, x0, y0, k, wy, wx)) {
            float s;
            const int g = halo_src_ty<TY>(S, x0, y0, wy * kHX + (wx - 2), s);
            if (s != 0.f) {  // zero-sign ghosts stay the zeros the copy filled in
              gcell[h] = wy * kWX + wx;
              gs[h] = s;
              gz[h] = f2{__ldg(z + g), __ldg(z_lo + g)};
              gp[h] = f2{__ldg(pold + g), __ldg(pold_lo + g)};
            }
          }
        }
      }
      mbar_wait(&full[b], (n_used >> 1) & 1, abort_flag, wait_cycles);
      // p = z + beta p_old over the whole window, in place of z
      float4* zh = reinterpret_cast<float4*>(buf);
      float4* zl = reinterpret_cast<float4*>(buf + G::kWinBytes);
      const float4* ph = reinterpret_cast<const float4*>(buf + 2 * G::kWinBytes);
      const float4* pl = reinterpret_cast<const float4*>(buf + 3 * G::kWinBytes);
      for (int v = threadIdx.x; v < kWX * G::kHYt / 4; v += kStThreads) {
        const float4 a = zh[v], al = zl[v], c = ph[v], cl = pl[v];
        const f2x2 u = df_axpy2(beta, {make_float2(c.x, c.y), make_float2(cl.x, cl.y)},
                                {make_float2(a.x, a.y), make_float2(al.x, al.y)});
        const f2x2 t = df_axpy2(beta, {make_float2(c.z, c.w), make_float2(cl.z, cl.w)},
                                {make_float2(a.z, a.w), make_float2(al.z, al.w)});
        zh[v] = make_float4(u.hi.x, u.hi.y, t.hi.x, t.hi.y);
        zl[v] = make_float4(u.lo.x, u.lo.y, t.lo.x, t.lo.y);
      }
      __syncthreads();
      if (*abort_flag) break;  // every thread reads the flag after the barrier: uniform
      ++n_used;
      if (!interior) {
        float* wh = reinterpret_cast<float*>(buf);
        float* wl = reinterpret_cast<float*>(buf + G::kWinBytes);
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (gcell[h] >= 0) {
            const f2 v = df_add(gz[h], df_mul(gp[h], beta));
            wh[gcell[h]] = gs[h] * v.hi;
            wl[gcell[h]] = gs[h] * v.lo;
          }
        __syncthreads();
      }
    } else {
      // plain loads into the free window set, kChunk cells per thread in flight at a time
      buf = sbuf + ((n_used + 1) & 1) * G::kBufBytes;
      float* wh = reinterpret_cast<float*>(buf);
      float* wl = reinterpret_cast<float*>(buf + G::kWinBytes);
      uint8_t* mt = buf + 4 * G::kWinBytes;
      for (int e = threadIdx.x; e < G::kMaskBytes; e += kStThreads) {
        const int ly = e / kStTileX, lx = e - ly * kStTileX;
        const int gx = x0 + lx, gy = y0 + ly;
        mt[e] = (gx < S.nx && gy < S.ny) ? S.mask[gy * S.nx + gx] : 0;
      }
      constexpr int kChunk = 4;
#pragma unroll 1
      for (int i0 = 0; i0 < G::kHalo; i0 += kChunk * kStThreads) {
        int gi[kChunk];
        float gsg[kChunk];
        f2 zv[kChunk], pv[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int i = i0 + threadIdx.x + j * kStThreads;
          gsg[j] = 0.f;
          gi[j] = 0;
          if (i < G::kHalo) gi[j] = halo_src_ty<TY>(S, x0, y0, i, gsg[j]);
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const bool on = gsg[j] != 0.f;
          zv[j] = on ? f2{__ldg(z + gi[j]), __ldg(z_lo + gi[j])} : f2{0.f, 0.f};
          pv[j] = on ? f2{__ldg(pold + gi[j]), __ldg(pold_lo + gi[j])} : f2{0.f, 0.f};
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int i = i0 + threadIdx.x + j * kStThreads;
          if (i < G::kHalo) {
            const int ly = i / kHX, lx = i - ly * kHX;
            const f2 v = df_add(zv[j], df_mul(pv[j], beta));
            wh[ly * kWX + lx + 2] = gsg[j] * v.hi;
            wl[ly * kWX + lx + 2] = gsg[j] * v.lo;
          }
        }
      }
      __syncthreads();
    }
    const float* wh = reinterpret_cast<const float*>(buf);
    const float* wl = reinterpret_cast<const float*>(buf + G::kWinBytes);
    const uint8_t* mt = buf + 4 * G::kWinBytes;
    float* __restrict__ qh = S.q;
    float* __restrict__ ql = S.q_lo;
    const int nbx = (S.nx + kStTileX - 1) / kStTileX;  // 64-node blocks per grid row
    // p.q of the tile's 64 x 16 blocks: each thread sums its nodes of one block in step order, the
    // warp its lanes in a fixed butterfly, and one thread the eight warps in order
    CompDotDF dot;
    if (!ANISO) {
      // node pairs (x, x+1): the window's row stride is even and x - x0 is even.  In step j the
      // warp covers one tile row; lanes 0-15 its first 32 nodes, lanes 16-31 the next 32.  Two
      // steps (eight rows each) make a 16-row block.
#pragma unroll 1
      for (int j = 0; j < G::kOwn / 2; ++j) {
        const int k = threadIdx.x + j * kStThreads;
        const int ly = k / (kStTileX / 2), lx = 2 * (k - ly * (kStTileX / 2));
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx < S.nx && gy < S.ny) {
          const int g = gy * S.nx + gx;
          const int wc = (ly + 2) * kWX + lx + 4;
          const float2 pvh = ld2(wh + wc), pvl = ld2(wl + wc);
          const unsigned m2 = *reinterpret_cast<const uint16_t*>(mt + ly * kStTileX + lx);
          f2x2 q2 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          if (m2) {
            const CompSum2 a = stencil13_pair_acc<kWX>(wh + wc);
            const float2 l = stencil13_pair_plain<kWX>(wl + wc);
            q2 = df_norm2(a.s, add2(a.c, l));
          }
          const bool m0 = (m2 & 0xffu) != 0, m1 = (m2 >> 8) != 0;
          const f2 q0 = m0 ? f2{q2.hi.x, q2.lo.x} : f2{0.f, 0.f};
          const f2 q1 = m1 ? f2{q2.hi.y, q2.lo.y} : f2{0.f, 0.f};
          dot.add(pvh.x, pvl.x, q0.hi, q0.lo);
          if (gx + 1 < S.nx) {
            dot.add(pvh.y, pvl.y, q1.hi, q1.lo);
            if ((g & 1) == 0) {
              *reinterpret_cast<float2*>(pnew + g) = pvh;
              *reinterpret_cast<float2*>(pnew_lo + g) = pvl;
              *reinterpret_cast<float2*>(qh + g) = make_float2(q0.hi, q1.hi);
              *reinterpret_cast<float2*>(ql + g) = make_float2(q0.lo, q1.lo);
            } else {
              pnew[g] = pvh.x;
              pnew[g + 1] = pvh.y;
              pnew_lo[g] = pvl.x;
              pnew_lo[g + 1] = pvl.y;
              qh[g] = q0.hi;
              qh[g + 1] = q1.hi;
              ql[g] = q0.lo;
              ql[g + 1] = q1.lo;
            }
          } else {
            pnew[g] = pvh.x;
            pnew_lo[g] = pvl.x;
            qh[g] = q0.hi;
            ql[g] = q0.lo;
          }
        }
        if (j & 1) {  // the end of a 16-row block: every lane joins the butterfly
          const double blk = group_sum_comp<32>(dot.s, dot.c);
          if (lane == 0) blk_sm[j >> 1][threadIdx.x >> 5] = blk;
          dot = CompDotDF{};
        }
      }
    } else {
      // one node per lane; in step j the warp covers 32 consecutive nodes of one tile row; four
      // steps (four rows each) make a 16-row block
#pragma unroll 1
      for (int j = 0; j < G::kOwn; ++j) {
        const int k = threadIdx.x + j * kStThreads;
        const int ly = k / kStTileX, lx = k - ly * kStTileX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx < S.nx && gy < S.ny) {
          const int g = gy * S.nx + gx;
          const float pvh = wh[(ly + 2) * kWX + lx + 4], pvl = wl[(ly + 2) * kWX + lx + 4];
          f2 qv = {0.f, 0.f};
          if (mt[ly * kStTileX + lx]) {
            const CompSum a = stencil13_acc<ANISO, kWX>(S, wh + 2, ly, lx);
            const float l = stencil13_plain<ANISO, kWX>(S, wl + 2, ly, lx);
            qv = df_norm(a.s, __fadd_rn(a.c, l));
          }
          pnew[g] = pvh;
          pnew_lo[g] = pvl;
          qh[g] = qv.hi;
          ql[g] = qv.lo;
          dot.add(pvh, pvl, qv.hi, qv.lo);
        }
        if ((j & 3) == 3) {
          const double blk = group_sum_comp<32>(dot.s, dot.c);
          if (lane == 0) blk_sm[j >> 2][threadIdx.x >> 5] = blk;
          dot = CompDotDF{};
        }
      }
    }
    __syncthreads();  // the window set is free for the copies started at the next copied tile
    // the 16-row blocks of the tile (TY / 16 of them, so the partials do not depend on TY); the
    // next tile writes blk_sm only after its own block barriers, which these threads join later
    if (threadIdx.x < TY / 16) {
      const int by = (y0 >> 4) + threadIdx.x;
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < kStThreads / 32; ++w) acc += blk_sm[threadIdx.x][w];
      if (16 * by < S.ny) S.pq_part[by * nbx + x0 / kStTileX] = acc;
    }
  }
  if (threadIdx.x == 0) {
    // copies still in flight (only after an abort) land before the block's memory is released
    for (int o = n_used; o < n_issued; ++o) {
      const long long t0 = clock64();
      while (!mbar_try(&full[o & 1], (o >> 1) & 1) && clock64() - t0 < kWaitCycles / 4) {
      }
    }
    if (s_abort) atomicExch(err, 1);
  }
}

// One block per slot (the slot's tile-0 item of the per-slot list): p.q from the stencil's
// block partials (64 x 16 nodes) in a fixed order, alpha = rho / p.q, breakdown detection.
__global__ void __launch_bounds__(256)
k_pq_finish(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
            const int* __restrict__ n_items) {
  __shared__ double red[64];
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    if (it.tile != 0) continue;
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    if (!sc->active) continue;
    double a = 0.0, b = 0.0;
    const int nparts = ((S.ny + 15) >> 4) * ((S.nx + kStTileX - 1) / kStTileX);
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) a += __ldcg(&S.pq_part[t]);
    block_sum2<256>(a, b, red);
    if (threadIdx.x == 0) {
      sc->pq = a;
      if (!(a > 0.0) || !isfinite(a) || !isfinite(sc->rho)) {
        sc->status = ST_EBREAKDOWN;
        sc->active = 0;
        sc->fold = 1;  // the tail replaces the residual and reports the best iterate
      } else {
        sc->alpha = sc->rho / a;
        const double aro = sc->alpha * sc->rho;
        sc->aro_total += aro;
        sc->aro_ring[sc->aro_n % kErrDelay] = aro;
        sc->aro_n += 1;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Iteration, stage 2: x += alpha p, r -= alpha q (all double-float), partial ||r||^2.  The last
// item advances the iteration count and decides stop / residual replacement.  Each thread moves
// 16-byte vectors (4 elements per access) of every plane; all loads are issued before any
// arithmetic.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecThreads)
k_update(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
         const int* __restrict__ n_items) {
  __shared__ double red[64];
  __shared__ int s_last;
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    if (!sc->active) continue;
    const f2 alpha = df_of(sc->alpha);
    const f2 nalpha = {-alpha.hi, -alpha.lo};
    const int pi = (sc->it & 1) ^ 1;
    const float* __restrict__ p = S.p[pi];
    const float* __restrict__ p_lo = S.p_lo[pi];
    const int n = S.nx * S.ny;
    const int e0 = it.tile * kVecChunk;
    const int e1 = min(n, e0 + kVecChunk);
    CompDotDF dot;
    constexpr int kStep = 4 * kVecThreads;
    constexpr int kVec = kVecChunk / kStep;
    if (e0 + kVecChunk <= n) {
      // full chunk: kU 16-byte vectors of every plane in flight per thread, loads first
      constexpr int kU = 2;
      static_assert(kVec % kU == 0, "unroll");
#pragma unroll 1
      for (int j0 = 0; j0 < kVec; j0 += kU) {
        float4 ph[kU], pl[kU], qh[kU], ql[kU], rh[kU], rl[kU], xh[kU], xl[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int e = e0 + (j0 + u) * kStep + 4 * threadIdx.x;
          ph[u] = __ldg(reinterpret_cast<const float4*>(p + e));
          pl[u] = __ldg(reinterpret_cast<const float4*>(p_lo + e));
          qh[u] = __ldg(reinterpret_cast<const float4*>(S.q + e));
          ql[u] = __ldg(reinterpret_cast<const float4*>(S.q_lo + e));
          rh[u] = *reinterpret_cast<const float4*>(S.r + e);
          rl[u] = *reinterpret_cast<const float4*>(S.r_lo + e);
          xh[u] = *reinterpret_cast<const float4*>(S.xhi + e);
          xl[u] = *reinterpret_cast<const float4*>(S.xlo + e);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int e = e0 + (j0 + u) * kStep + 4 * threadIdx.x;
          df_axpy(xh[u].x, xl[u].x, alpha, ph[u].x, pl[u].x);
          df_axpy(xh[u].y, xl[u].y, alpha, ph[u].y, pl[u].y);
          df_axpy(xh[u].z, xl[u].z, alpha, ph[u].z, pl[u].z);
          df_axpy(xh[u].w, xl[u].w, alpha, ph[u].w, pl[u].w);
          df_axpy(rh[u].x, rl[u].x, nalpha, qh[u].x, ql[u].x);
          df_axpy(rh[u].y, rl[u].y, nalpha, qh[u].y, ql[u].y);
          df_axpy(rh[u].z, rl[u].z, nalpha, qh[u].z, ql[u].z);
          df_axpy(rh[u].w, rl[u].w, nalpha, qh[u].w, ql[u].w);
          *reinterpret_cast<float4*>(S.xhi + e) = xh[u];
          *reinterpret_cast<float4*>(S.xlo + e) = xl[u];
          *reinterpret_cast<float4*>(S.r + e) = rh[u];
          *reinterpret_cast<float4*>(S.r_lo + e) = rl[u];
          dot.add(rh[u].x, rl[u].x, rh[u].x, rl[u].x);
          dot.add(rh[u].y, rl[u].y, rh[u].y, rl[u].y);
          dot.add(rh[u].z, rl[u].z, rh[u].z, rl[u].z);
          dot.add(rh[u].w, rl[u].w, rh[u].w, rl[u].w);
        }
      }
    } else {
      for (int k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
        float xh = S.xhi[k], xl = S.xlo[k];
        df_axpy(xh, xl, alpha, p[k], p_lo[k]);
        S.xhi[k] = xh;
        S.xlo[k] = xl;
        float rh = S.r[k], rl = S.r_lo[k];
        df_axpy(rh, rl, nalpha, S.q[k], S.q_lo[k]);
        S.r[k] = rh;
        S.r_lo[k] = rl;
        dot.add(rh, rl, rh, rl);
      }
    }
    const double rr = block_sum_comp<kVecThreads>(dot.as_comp(), red);
    if (threadIdx.x == 0) S.part[it.tile * 4 + 0] = rr;
    if (last_item_block(&sc->cnt[2], S.n_vec_items, &s_last)) {
      double sums[1];
      reduce_partials<kVecThreads, 1>(S.part, S.n_vec_items, sums, red);
      if (threadIdx.x == 0) {
        const double s = sums[0];
        sc->rr = s;
        const int itn = sc->it + 1;
        sc->it = itn;
        if (s <= sc->rtol2 * sc->bb || itn >= sc->maxit || !isfinite(s)) {
          sc->active = 0;
          sc->fold = 1;
        } else if (s < sc->delta2 * sc->rr_ref || itn % sc->fold_every == 0) {
          sc->fold = 1;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Tail: true residual r = b - M L^2 xhat in FP64, replace the recursive residual, and decide:
// converged / not converged at maxit / continue (with a fresh preconditioner pass).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kStThreads)
k_true_residual(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
                const int* __restrict__ n_items) {
  __shared__ double sx[kHalo];
  __shared__ double red[64];
  __shared__ int s_last;
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    if (!sc->fold) continue;
    const int be = sc->bexp;
    int x0, y0;
    tile_origin(S, it.tile, x0, y0);
    for (int i = threadIdx.x; i < kHalo; i += blockDim.x) {
      float s;
      const int g = halo_src(S, x0, y0, i, s);
      sx[i] = (s != 0.f) ? (double)s * ((double)S.xhi[g] + (double)S.xlo[g]) : 0.0;
    }
    __syncthreads();
    double rr = 0.0;
    for (int k = threadIdx.x; k < kStTileX * kStTileY; k += blockDim.x) {
      const int ly = k / kStTileX, lx = k - ly * kStTileX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx >= S.nx || gy >= S.ny) continue;
      const int g = gy * S.nx + gx;
      double rv = 0.0;
      if (S.mask[g]) rv = ldexp(S.b[g], be) - stencil13_f64(S, sx, ly, lx);
      const f2 v = df_of(rv);
      S.r[g] = v.hi;
      S.r_lo[g] = v.lo;
      rr += rv * rv;
    }
    double d2 = 0.0;
    block_sum2<kStThreads>(rr, d2, red);
    if (threadIdx.x == 0) S.part[it.tile * 4 + 0] = rr;
    if (last_item_block(&sc->cnt[3], S.n_st_tiles, &s_last)) {
      double sums[1];
      reduce_partials<kStThreads, 1>(S.part, S.n_st_tiles, sums, red);
      if (threadIdx.x == 0) {
        const double s = sums[0];
        sc->rr_true = s;
        sc->rr = s;
        sc->rr_ref = s;
        sc->fold = 0;
        if (sc->status == ST_EBREAKDOWN) {
          sc->active = 0;
          sc->need_prec = 0;
          if (s <= sc->rtol2 * sc->bb) sc->status = ST_OK;
        } else if (s <= sc->rtol2 * sc->bb) {
          sc->status = ST_OK;
          sc->active = 0;
          sc->need_prec = 0;
        } else if (sc->it >= sc->maxit || !isfinite(s)) {
          sc->status = ST_ENOTCONV;
          sc->active = 0;
          sc->need_prec = 0;
        } else {
          sc->active = 1;
          sc->need_prec = 1;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// After the last preconditioner stage: one block per slot (the slot's tile-0 item of the
// transform work list) reduces the per-tile r.z and z.q partials in a fixed order and forms rho
// and beta (flexible or Fletcher-Reeves), or flags breakdown.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_prec_finish(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
              const int* __restrict__ n_items, int mode) {
  __shared__ double red[64];
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    if (it.tile != 0) continue;
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    const int run = mode == 0 ? sc->active : (mode == 1 ? sc->need_prec : 1);
    if (!run) continue;
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < S.n_prec_parts; t += blockDim.x) {
      a += S.part[t * 4 + 2];
      b += S.part[t * 4 + 3];
    }
    block_sum2<256>(a, b, red);
    if (threadIdx.x == 0) finish_preconditioner(S, a, b, mode);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Output (Algorithm 1, last statement): out = f at known nodes (bit copy), xhat at unknowns.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecThreads)
k_output(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
         const int* __restrict__ n_items, const float* const* __restrict__ fs,
         float* const* __restrict__ outs) {
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    const float* f = fs[it.slot];
    float* out = outs[it.slot];
    const int n = S.nx * S.ny;
    const int e0 = it.tile * kVecChunk;
    const int e1 = min(n, e0 + kVecChunk);
    const int be = S.sc->bexp;  // x = 2^-bexp x'
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x)
      out[e] = S.mask[e] ? (float)ldexp((double)S.xhi[e] + (double)S.xlo[e], -be) : f[e];
  }
}

// FP64 variant of the output for one slot (lets the caller recompute the residual exactly).
__global__ void __launch_bounds__(kVecThreads)
k_output64(const SlotDesc* __restrict__ slots, const float* __restrict__ f, double* __restrict__ out) {
  const SlotDesc& S = slots[0];
  const int n = S.nx * S.ny;
  const int be = S.sc->bexp;  // x = 2^-bexp x'
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    out[e] = S.mask[e] ? ldexp((double)S.xhi[e] + (double)S.xlo[e], -be) : (double)f[e];
}

// ---------------------------------------------------------------------------------------------
// q = M L^2 p for a caller-supplied FP32 p (same compensated evaluation, one node per thread;
// used by the entry point that allocates nothing).
// ---------------------------------------------------------------------------------------------
template <bool ANISO>
__global__ void __launch_bounds__(kStThreads)
k_apply(const SlotDesc* __restrict__ slots, const float* __restrict__ p, float* __restrict__ q,
        double* __restrict__ part) {
  __shared__ float sp[kHalo];
  __shared__ double red[64];
  const SlotDesc& S = slots[0];
  for (int tile = blockIdx.x; tile < S.n_st_tiles; tile += gridDim.x) {
    int x0, y0;
    tile_origin(S, tile, x0, y0);
    for (int i = threadIdx.x; i < kHalo; i += blockDim.x) {
      float s;
      const int g = halo_src(S, x0, y0, i, s);
      sp[i] = (s != 0.f) ? s * p[g] : 0.f;
    }
    __syncthreads();
    double pq = 0.0;
    for (int k = threadIdx.x; k < kStTileX * kStTileY; k += blockDim.x) {
      const int ly = k / kStTileX, lx = k - ly * kStTileX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx >= S.nx || gy >= S.ny) continue;
      const int g = gy * S.nx + gx;
      float qv = 0.f;
      if (S.mask[g]) qv = stencil13<ANISO>(S, sp, ly, lx);
      q[g] = qv;
      pq += (double)p[g] * (double)qv;
    }
    double d2 = 0.0;
    block_sum2<kStThreads>(pq, d2, red);
    if (threadIdx.x == 0) part[tile] = pq;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------
void launch_setup(const LaunchCfg& c, const float* const* phis, const float* const* fs,
                  const int* dirs) {
  k_setup<<<c.grid, kStThreads, 0, c.stream>>>(c.slots, c.items, c.n_items, phis, fs, dirs);
}
void launch_rhs_scale(const LaunchCfg& c) {
  k_rhs_scale<<<c.grid, kStThreads, 0, c.stream>>>(c.slots, c.items, c.n_items);
}
template <int TY>
static void launch_stencil_ty(const LaunchCfg& c, bool aniso, int* err, long long wc) {
  constexpr int smem = StGeom<TY>::kSmemBytes;
  if (aniso)
    k_stencil<true, TY><<<c.grid, kStThreads, smem, c.stream>>>(c.slots, c.items, c.n_items, err, wc);
  else
    k_stencil<false, TY><<<c.grid, kStThreads, smem, c.stream>>>(c.slots, c.items, c.n_items, err, wc);
}
void launch_stencil(const LaunchCfg& c, bool aniso, int tile_y, int* err) {
  const long long wc = c.wait_cycles > 0 ? c.wait_cycles : kWaitCycles;
  if (tile_y == 16) launch_stencil_ty<16>(c, aniso, err, wc);
  else launch_stencil_ty<32>(c, aniso, err, wc);
}
int stencil_blocks_per_sm(int tile_y) {
  return tile_y == 16 ? StGeom<16>::kBlocksPerSm : StGeom<32>::kBlocksPerSm;
}
template <bool ANISO, int TY>
static cudaError_t stencil_attr() {
  // the window sets live in dynamic shared memory; all of the SM's shared memory to the
  // carveout, so that kBlocksPerSm blocks fit
  const cudaError_t e = cudaFuncSetAttribute(k_stencil<ANISO, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             StGeom<TY>::kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_stencil<ANISO, TY>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}
cudaError_t stencil_init() {
  const cudaError_t e[4] = {stencil_attr<false, 32>(), stencil_attr<true, 32>(),
                            stencil_attr<false, 16>(), stencil_attr<true, 16>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}
void launch_pq_finish(const LaunchCfg& c) {
  k_pq_finish<<<c.grid, 256, 0, c.stream>>>(c.slots, c.items, c.n_items);
}
void launch_update(const LaunchCfg& c) {
  k_update<<<c.grid, kVecThreads, 0, c.stream>>>(c.slots, c.items, c.n_items);
}
void launch_true_residual(const LaunchCfg& c) {
  k_true_residual<<<c.grid, kStThreads, 0, c.stream>>>(c.slots, c.items, c.n_items);
}
void launch_output(const LaunchCfg& c, const float* const* fs, float* const* outs) {
  k_output<<<c.grid, kVecThreads, 0, c.stream>>>(c.slots, c.items, c.n_items, fs, outs);
}
void launch_prec_finish(const LaunchCfg& c, int mode) {
  k_prec_finish<<<c.grid, 256, 0, c.stream>>>(c.slots, c.items, c.n_items, mode);
}
void launch_output64(const SlotDesc* slot, int n, const float* f, double* out, cudaStream_t s) {
  int grid = (n + kVecThreads - 1) / kVecThreads;
  grid = grid < 4096 ? grid : 4096;
  k_output64<<<grid, kVecThreads, 0, s>>>(slot, f, out);
}
void launch_apply(const SlotDesc* slot, int n_tiles, bool aniso, const float* p, float* q,
                  double* part, cudaStream_t s) {
  const int grid = n_tiles < 4096 ? n_tiles : 4096;
  if (aniso) k_apply<true><<<grid, kStThreads, 0, s>>>(slot, p, q, part);
  else k_apply<false><<<grid, kStThreads, 0, s>>>(slot, p, q, part);
}

}  // namespace bx
