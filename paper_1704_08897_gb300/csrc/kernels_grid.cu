// Grid kernels of the PCG extension solve: right-hand side, masked biharmonic apply, CG vector
// update, residual replacement and output.  All are persistent launches over a work list of
// (slot, tile) items so that one launch serves a single solve, a batch or the serving loop.
//
// The operator is eq. (discrete_biharmonic) of Sec. 2.1 with the boundary rules of Algorithm 1
// (Dirichlet padding), half-sample reflection (symmetric) or wrap-around (periodic), evaluated
// matrix-free ("no need to form the 13-banded matrix", Sec. 2.2).
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

// 13-point masked biharmonic of a smem tile (row stride RS) at local (ly+2, lx+2), compensated
// FP32.
template <bool ANISO, int RS = kHX>
__device__ __forceinline__ float stencil13(const SlotDesc& S, const float* t, int ly, int lx) {
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
  return acc.result();
}

// The isotropic 13-point stencil at two adjacent nodes (x, x+1) of a smem tile with an even row
// stride RS; c points at node x, an even index.  Eleven aligned 8-byte loads cover both
// neighbourhoods, and each lane runs the scalar stencil13's operations in the same order
// (bit-identical results).
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
template <int RS>
__device__ __forceinline__ float2 stencil13_pair(const float* c) {
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
  return acc.result();
}

__device__ __forceinline__ double stencil13_f64(const SlotDesc& S, const double* t, int ly, int lx) {
  const double* c = t + (ly + 2) * kHX + (lx + 2);
  return S.dwc * c[0] + S.dwex * (c[-1] + c[1]) + S.dwey * (c[-kHX] + c[kHX]) +
         S.dwd * ((c[-kHX - 1] + c[-kHX + 1]) + (c[kHX - 1] + c[kHX + 1])) +
         S.dwfx * (c[-2] + c[2]) + S.dwfy * (c[-2 * kHX] + c[2 * kHX]);
}

// ---------------------------------------------------------------------------------------------
// Setup: known mask from sign(phi) (Sec. 2.1), b = -M L^2 E_K f in FP64 (Algorithm 1, first
// statement), zero CG state.  Partials: ||b||^2, number of known nodes, number of NaN phi.
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
    double bb = 0.0, cnt = 0.0, nan = 0.0;
    for (int k = threadIdx.x; k < kStTileX * kStTileY; k += blockDim.x) {
      const int ly = k / kStTileX, lx = k - ly * kStTileX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx >= S.nx || gy >= S.ny) continue;
      const int g = gy * S.nx + gx;
      const float ph = phi[g];
      const bool known = out_dir ? (ph < 0.f) : (ph > 0.f);
      if (ph != ph) nan += 1.0;
      double bv = 0.0;
      if (!known) bv = -stencil13_f64(S, sf, ly, lx);
      S.mask[g] = known ? 0 : 1;
      S.b[g] = bv;
      S.xhi[g] = 0.f;
      S.xlo[g] = 0.f;
      S.r[g] = (float)bv;
      S.p[0][g] = 0.f;
      S.p[1][g] = 0.f;
      S.q[g] = 0.f;
      S.z[g] = 0.f;
      bb += bv * bv;
      cnt += known ? 1.0 : 0.0;
    }
    block_sum2<kStThreads>(bb, cnt, red);
    double nn = nan, dummy = 0.0;
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
        if (sn > 0.0) {
          sc->status = -1;  // EXT_EINVAL: NaN in phi
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

// Set-up, second pass: r = 2^e b in FP32, once the slot's scale exponent e is known.
__global__ void __launch_bounds__(kStThreads)
k_rhs_scale(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
            const int* __restrict__ n_items) {
  const int total = *n_items;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    const int e = S.sc->bexp;
    int x0, y0;
    tile_origin(S, it.tile, x0, y0);
    for (int k = threadIdx.x; k < kStTileX * kStTileY; k += blockDim.x) {
      const int ly = k / kStTileX, lx = k - ly * kStTileX;
      const int gx = x0 + lx, gy = y0 + ly;
      if (gx >= S.nx || gy >= S.ny) continue;
      const int g = gy * S.nx + gx;
      S.r[g] = (float)ldexp(S.b[g], e);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Iteration, stage 1: p = z + beta p_old (formed in shared memory including the halo),
// q = M L^2 p (Algorithm 1, matvec, with the mask in the epilogue), per-tile partial p.q;
// k_pq_finish then forms alpha = rho / p.q for each slot.
//
// Each block walks its share of the (slot, tile) list with two shared-memory windows.  For a slot
// whose rows span a multiple of 16 bytes in the mask (nx % 16 == 0), the window of the block's
// next tile arrives by tensor copies while it computes the current one: z and p_old over rows
// y0-2 .. y0+33 and columns x0-4 .. x0+67 (two columns wider on the left than the halo, so that
// each copy starts on a 16-byte boundary) and the tile's mask bytes.  Cells outside the grid
// arrive as zeros; the ghost cells of a boundary tile (reflected, wrapped or negated copies of
// grid nodes under the boundary rule) are gathered by plain loads.  Tiles of other slots fill the
// free window with plain loads.
// ---------------------------------------------------------------------------------------------
constexpr int kWX = kStWinX;                           // 72: window row, floats
static_assert(kStWinY == kHY, "the window spans the halo rows");
constexpr int kWinBytes = kWX * kHY * 4;               // one float window (z, then p; p_old)
constexpr int kMaskBytes = kStTileX * kStTileY;        // the tile's mask
constexpr int kBufBytes = 2 * kWinBytes + kMaskBytes;  // one window set
static_assert(kWinBytes % 128 == 0 && kBufBytes % 128 == 0, "tensor copy destinations");
constexpr int kGhostSlots = 4 * kHY + 4 * kHX;         // candidate ghost cells of one halo
static_assert(kGhostSlots <= 2 * kStThreads, "two ghost candidates per thread");
constexpr int kStBlocksPerSm = 4;

// Candidate k of a tile's ghost cells: the four ghost columns (x = -2, -1, nx, nx+1) over the
// halo's rows, then the four ghost rows over the halo's in-grid columns.  Returns false when the
// candidate lies outside the halo or beyond the second ghost line; (wy, wx) is its window cell.
__device__ __forceinline__ bool ghost_cell(const SlotDesc& S, int x0, int y0, int k, int& wy,
                                           int& wx) {
  if (k < 4 * kHY) {
    const int j = k / kHY;
    wy = k - j * kHY;
    const int gx = j < 2 ? j - 2 : S.nx + (j - 2);
    const int lx = gx - (x0 - 2);
    wx = lx + 2;
    return lx >= 0 && lx < kHX && y0 - 2 + wy <= S.ny + 1;
  }
  const int kk = k - 4 * kHY;
  const int j = kk / kHX, lx = kk - j * kHX;
  const int gy = j < 2 ? j - 2 : S.ny + (j - 2);
  const int gx = x0 - 2 + lx;
  wy = gy - (y0 - 2);
  wx = lx + 2;
  return wy >= 0 && wy < kHY && gx >= 0 && gx < S.nx;
}

// Thread 0: start the tensor copies of the block's next copied tile (the next item at or after
// w_issue whose slot iterates and has stencil maps) into window set n_issued % 2.
__device__ __forceinline__ void stencil_issue_next(const SlotDesc* __restrict__ slots,
                                                   const WorkItem* __restrict__ items, int total,
                                                   unsigned char (*sbuf)[kBufBytes],
                                                   uint64_t* full, int& w_issue, int& n_issued) {
  while (w_issue < total) {
    const WorkItem it = items[w_issue];
    w_issue += gridDim.x;
    const SlotDesc& S = slots[it.slot];
    if (S.st_maps == nullptr || !S.sc->active) continue;
    int x0, y0;
    tile_origin(S, it.tile, x0, y0);
    const unsigned char* maps = static_cast<const unsigned char*>(S.st_maps);
    const void* mz = maps;
    const void* mp = maps + 128 * (1 + (S.sc->it & 1));
    const void* mm = maps + 128 * 3;
    tmap_acquire(mz);
    tmap_acquire(mp);
    tmap_acquire(mm);
    const int b = n_issued & 1;
    unsigned char* dst = sbuf[b];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&full[b], kBufBytes);
    tma_load_2d(dst, mz, &full[b], x0 - 4, y0 - 2);
    tma_load_2d(dst + kWinBytes, mp, &full[b], x0 - 4, y0 - 2);
    tma_load_2d(dst + 2 * kWinBytes, mm, &full[b], x0, y0);
    ++n_issued;
    return;
  }
}

template <bool ANISO>
__global__ void __launch_bounds__(kStThreads, kStBlocksPerSm)
k_stencil(const SlotDesc* __restrict__ slots, const WorkItem* __restrict__ items,
          const int* __restrict__ n_items, int* __restrict__ err) {
  __shared__ __align__(128) unsigned char sbuf[2][kBufBytes];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ double red[64];
  __shared__ int s_abort;
  const int total = *n_items;
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
  if (threadIdx.x == 0) stencil_issue_next(slots, items, total, sbuf, full, w_issue, n_issued);
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const WorkItem it = items[w];
    const SlotDesc& S = slots[it.slot];
    SlotScalars* sc = S.sc;
    if (!sc->active) continue;
    const float beta = (float)sc->beta;
    const int par = sc->it & 1;
    const float* __restrict__ pold = S.p[par];
    float* __restrict__ pnew = S.p[par ^ 1];
    const float* __restrict__ z = S.z;
    int x0, y0;
    tile_origin(S, it.tile, x0, y0);
    // a tile whose halo lies inside the grid has no ghost cell
    const bool interior =
        x0 >= 2 && y0 >= 2 && x0 + kStTileX + 2 <= S.nx && y0 + kStTileY + 2 <= S.ny;
    unsigned char* buf;
    if (S.st_maps != nullptr) {
      const int b = n_used & 1;
      buf = sbuf[b];
      // the other window set finished with the previous tile: start the next tile's copies
      if (threadIdx.x == 0 && n_issued == n_used + 1)
        stencil_issue_next(slots, items, total, sbuf, full, w_issue, n_issued);
      // ghost cells by plain loads, issued before the wait so that both latencies overlap
      int gcell[2] = {-1, -1};
      float gz[2] = {0.f, 0.f}, gp[2] = {0.f, 0.f}, gs[2] = {0.f, 0.f};
      if (!interior) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = threadIdx.x + h * kStThreads;
          int wy, wx;
          if (k < kGhostSlots && ghost_cell(S, x0, y0, k, wy, wx)) {
            float s;
            const int g = halo_src(S, x0, y0, wy * kHX + (wx - 2), s);
            if (s != 0.f) {  // zero-sign ghosts stay the zeros the copy filled in
              gcell[h] = wy * kWX + wx;
              gs[h] = s;
              gz[h] = __ldg(z + g);
              gp[h] = __ldg(pold + g);
            }
          }
        }
      }
      mbar_wait(&full[b], (n_used >> 1) & 1, abort_flag);
      // p = z + beta p_old over the whole window, in place of z
      float4* zw = reinterpret_cast<float4*>(buf);
      const float4* pw = reinterpret_cast<const float4*>(buf + kWinBytes);
      for (int v = threadIdx.x; v < kWX * kHY / 4; v += kStThreads) {
        const float4 a = zw[v], c = pw[v];
        zw[v] = make_float4(__fmaf_rn(beta, c.x, a.x), __fmaf_rn(beta, c.y, a.y),
                            __fmaf_rn(beta, c.z, a.z), __fmaf_rn(beta, c.w, a.w));
      }
      __syncthreads();
      if (*abort_flag) break;  // every thread reads the flag after the barrier: uniform
      ++n_used;
      if (!interior) {
        float* wf = reinterpret_cast<float*>(buf);
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (gcell[h] >= 0) wf[gcell[h]] = gs[h] * __fmaf_rn(beta, gp[h], gz[h]);
        __syncthreads();
      }
    } else {
      // plain loads into the free window set, kChunk cells per thread in flight at a time
      buf = sbuf[(n_used + 1) & 1];
      float* wf = reinterpret_cast<float*>(buf);
      uint8_t* mt = buf + 2 * kWinBytes;
      for (int e = threadIdx.x; e < kMaskBytes; e += kStThreads) {
        const int ly = e / kStTileX, lx = e - ly * kStTileX;
        const int gx = x0 + lx, gy = y0 + ly;
        mt[e] = (gx < S.nx && gy < S.ny) ? S.mask[gy * S.nx + gx] : 0;
      }
      constexpr int kChunk = 4;
#pragma unroll 1
      for (int i0 = 0; i0 < kHalo; i0 += kChunk * kStThreads) {
        int gi[kChunk];
        float gsg[kChunk], zv[kChunk], pv[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int i = i0 + threadIdx.x + j * kStThreads;
          gsg[j] = 0.f;
          gi[j] = 0;
          if (i < kHalo) gi[j] = halo_src(S, x0, y0, i, gsg[j]);
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          zv[j] = gsg[j] != 0.f ? __ldg(z + gi[j]) : 0.f;
          pv[j] = gsg[j] != 0.f ? __ldg(pold + gi[j]) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int i = i0 + threadIdx.x + j * kStThreads;
          if (i < kHalo) {
            const int ly = i / kHX, lx = i - ly * kHX;
            wf[ly * kWX + lx + 2] = gsg[j] * __fmaf_rn(beta, pv[j], zv[j]);
          }
        }
      }
      __syncthreads();
    }
    const float* wf = reinterpret_cast<const float*>(buf);
    const uint8_t* mt = buf + 2 * kWinBytes;
    constexpr int kOwn = kStTileX * kStTileY / kStThreads;
    static_assert(kOwn * kStThreads == kStTileX * kStTileY && kOwn % 2 == 0, "tile / block size");
    CompDot dot;
    if (!ANISO) {
      // node pairs (x, x+1): the window's row stride is even and x - x0 is even
#pragma unroll 1
      for (int j = 0; j < kOwn / 2; ++j) {
        const int k = threadIdx.x + j * kStThreads;
        const int ly = k / (kStTileX / 2), lx = 2 * (k - ly * (kStTileX / 2));
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= S.nx || gy >= S.ny) continue;
        const int g = gy * S.nx + gx;
        const float* c = wf + (ly + 2) * kWX + lx + 4;
        const float2 pv = ld2(c);
        const unsigned m2 = *reinterpret_cast<const uint16_t*>(mt + ly * kStTileX + lx);
        const float2 q2 = m2 ? stencil13_pair<kWX>(c) : make_float2(0.f, 0.f);
        const float q0 = (m2 & 0xffu) ? q2.x : 0.f;
        const float q1 = (m2 >> 8) ? q2.y : 0.f;
        dot.add(pv.x, q0);
        if (gx + 1 < S.nx) {
          dot.add(pv.y, q1);
          if ((g & 1) == 0) {
            *reinterpret_cast<float2*>(pnew + g) = pv;
            *reinterpret_cast<float2*>(S.q + g) = make_float2(q0, q1);
          } else {
            pnew[g] = pv.x;
            pnew[g + 1] = pv.y;
            S.q[g] = q0;
            S.q[g + 1] = q1;
          }
        } else {
          pnew[g] = pv.x;
          S.q[g] = q0;
        }
      }
    } else {
#pragma unroll 1
      for (int j = 0; j < kOwn; ++j) {
        const int k = threadIdx.x + j * kStThreads;
        const int ly = k / kStTileX, lx = k - ly * kStTileX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= S.nx || gy >= S.ny) continue;
        const int g = gy * S.nx + gx;
        const float pv = wf[(ly + 2) * kWX + lx + 4];
        float qv = 0.f;
        if (mt[ly * kStTileX + lx]) qv = stencil13<ANISO, kWX>(S, wf + 2, ly, lx);
        pnew[g] = pv;
        S.q[g] = qv;
        dot.add(pv, qv);
      }
    }
    const double pq = block_sum_comp<kStThreads>(dot, red);
    if (threadIdx.x == 0) S.part[it.tile * 4 + 1] = pq;  // reduced by k_pq_finish
    __syncthreads();  // the window set is free for the copies started at the next copied tile
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

// One block per slot (the slot's tile-0 stencil item): p.q from the stencil's per-tile partials
// in a fixed order, alpha = rho / p.q, breakdown detection.
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
    for (int t = threadIdx.x; t < S.n_st_tiles; t += blockDim.x) a += S.part[t * 4 + 1];
    block_sum2<256>(a, b, red);
    if (threadIdx.x == 0) {
      sc->pq = a;
      if (!(a > 0.0) || !isfinite(a) || !isfinite(sc->rho)) {
        sc->status = ST_EBREAKDOWN;
        sc->active = 0;
        sc->fold = 1;  // the tail replaces the residual and reports the best iterate
      } else {
        sc->alpha = sc->rho / a;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Iteration, stage 2: x += alpha p (double-float), r -= alpha q (FP32), partial ||r||^2.  The
// last item advances the iteration count and decides stop / residual replacement.
// The iterate must carry more than FP32: an FP32 increment carries rounding errors of size
// eps |x|, which for this operator pin the true residual near 1e-6 while the recursive one
// keeps falling.  Each thread moves 16-byte vectors (4 elements per access).
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
    const float alpha = (float)sc->alpha;
    const float* __restrict__ p = S.p[(sc->it & 1) ^ 1];
    const int n = S.nx * S.ny;
    const int e0 = it.tile * kVecChunk;
    const int e1 = min(n, e0 + kVecChunk);
    CompDot dot;
    constexpr int kStep = 4 * kVecThreads;
    constexpr int kVec = kVecChunk / kStep;
    if (e0 + kVecChunk <= n) {
      // full chunk: issue every load of the thread before any arithmetic
      float4 pv[kVec], qv[kVec], rv[kVec], xh[kVec], xl[kVec];
#pragma unroll
      for (int j = 0; j < kVec; ++j) {
        const int e = e0 + j * kStep + 4 * threadIdx.x;
        pv[j] = __ldg(reinterpret_cast<const float4*>(p + e));
        qv[j] = __ldg(reinterpret_cast<const float4*>(S.q + e));
        rv[j] = *reinterpret_cast<const float4*>(S.r + e);
        xh[j] = *reinterpret_cast<const float4*>(S.xhi + e);
        xl[j] = *reinterpret_cast<const float4*>(S.xlo + e);
      }
#pragma unroll
      for (int j = 0; j < kVec; ++j) {
        const int e = e0 + j * kStep + 4 * threadIdx.x;
        df_axpy(xh[j].x, xl[j].x, alpha, pv[j].x);
        df_axpy(xh[j].y, xl[j].y, alpha, pv[j].y);
        df_axpy(xh[j].z, xl[j].z, alpha, pv[j].z);
        df_axpy(xh[j].w, xl[j].w, alpha, pv[j].w);
        rv[j].x = __fmaf_rn(-alpha, qv[j].x, rv[j].x);
        rv[j].y = __fmaf_rn(-alpha, qv[j].y, rv[j].y);
        rv[j].z = __fmaf_rn(-alpha, qv[j].z, rv[j].z);
        rv[j].w = __fmaf_rn(-alpha, qv[j].w, rv[j].w);
        *reinterpret_cast<float4*>(S.xhi + e) = xh[j];
        *reinterpret_cast<float4*>(S.xlo + e) = xl[j];
        *reinterpret_cast<float4*>(S.r + e) = rv[j];
        dot.add(rv[j].x, rv[j].x);
        dot.add(rv[j].y, rv[j].y);
        dot.add(rv[j].z, rv[j].z);
        dot.add(rv[j].w, rv[j].w);
      }
    } else {
      for (int k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
        float xh = S.xhi[k], xl = S.xlo[k];
        df_axpy(xh, xl, alpha, p[k]);
        S.xhi[k] = xh;
        S.xlo[k] = xl;
        const float rv = __fmaf_rn(-alpha, S.q[k], S.r[k]);
        S.r[k] = rv;
        dot.add(rv, rv);
      }
    }
    const double rr = block_sum_comp<kVecThreads>(dot, red);
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
// Tail: true residual r = b - M L^2 xhat in FP64, replace the recursive residual, and decide: converged / not converged at maxit / continue (with a fresh preconditioner pass).
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
      S.r[g] = (float)rv;
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
    for (int t = threadIdx.x; t < S.n_gm_tiles; t += blockDim.x) {
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
// Verification entry: q = M L^2 p for a caller-supplied p (same compensated evaluation).
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
void launch_stencil(const LaunchCfg& c, bool aniso, int* err) {
  if (aniso) k_stencil<true><<<c.grid, kStThreads, 0, c.stream>>>(c.slots, c.items, c.n_items, err);
  else k_stencil<false><<<c.grid, kStThreads, 0, c.stream>>>(c.slots, c.items, c.n_items, err);
}
int stencil_blocks_per_sm() { return kStBlocksPerSm; }
cudaError_t stencil_init() {
  // all of the SM's shared memory to the carveout, so that kStBlocksPerSm window pairs fit
  cudaError_t e = cudaFuncSetAttribute(k_stencil<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
  const cudaError_t e2 = cudaFuncSetAttribute(k_stencil<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              cudaSharedmemCarveoutMaxShared);
  return e != cudaSuccess ? e : e2;
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
