// Shared device-side definitions of the biharmonic extension library.
//
// One "slot" is one extension problem being solved; a batch (or the serving loop) is a set of
// slots.  Every CG stage is one launch over a work list of (slot, tile) items drawn from all
// iterating slots; per-slot scalars live in device memory and are reduced deterministically by
// the last work item of the slot to finish (fixed order, no floating-point atomics).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bx {

constexpr int kPad = 128;           // transform buffers are padded to multiples of this
constexpr int kStTileX = 64;        // stencil tile (x contiguous)
constexpr int kStTileY = 32;
constexpr int kStThreads = 256;
// The stencil's shared-memory window of one tile (also the box of its tensor copies): the halo
// rows y0-2 .. y0+kStTileY+1 and the columns x0-4 .. x0+kStTileX+3, two columns wider on the
// left than the halo so that a copy starts on a 16-byte boundary.
constexpr int kStWinX = kStTileX + 8;
constexpr int kStWinY = kStTileY + 4;
constexpr int kStMaps = 7;          // stencil tensor maps per slot
constexpr int kLowM = 32;           // low modes per axis computed in high precision
constexpr int kLowAutoSide = 2048;  // low_modes = 2: grids with a side of at least this many nodes
constexpr long long kLowAutoNodes = 2048LL * 2048;  // low_modes = 2: or calls with this many nodes
constexpr int kLowNS = 6;           // integer slices per operand of the low-mode products
constexpr int kLowK3 = 64;          // k extent of the inverse low-mode product (32 modes, zero-padded)
constexpr int kVecChunk = 4096;     // elements per work item of the vector kernels
constexpr int kVecThreads = 256;

enum Bc : int { BC_SYM = 0, BC_PER = 1, BC_DIR = 2 };

// Status words (match the public EXT_* codes).
enum : int { ST_OK = 0, ST_RUNNING = 1, ST_ENOTCONV = -5, ST_EBREAKDOWN = -6 };

// Per-slot scalars, FP64 where they feed CG.  Written only by the last work item of a slot.
struct __align__(16) SlotScalars {
  double bb;        // ||b||^2
  double rho;       // r.z of the current z
  double pq;        // p.Ap of the current direction
  double zq;        // z_new.q_old (flexible beta)
  double rr;        // ||r||^2, recursive
  double rr_true;   // ||b - A xhat||^2 at the last replacement
  double alpha, beta;
  double rtol2;     // rtol^2
  double rr_ref;    // ||r||^2 at the last residual replacement
  double delta2;    // replace the residual once ||r||^2 < delta2 * rr_ref
  int it;           // completed iterations
  int maxit;
  int fold_every;   // longest stretch of iterations between residual replacements
  int active;       // 1 while the slot iterates
  int fold;         // 1: the tail replaces r by the FP64 true residual b - A xhat
  int need_prec;    // 1: the tail preconditioner runs (after a replacement that continues)
  int status;       // ST_RUNNING until final
  int flexible;
  unsigned cnt[6];  // completion counters of the last-item reductions, one per kernel kind
  int n_known;      // known nodes, counted by the set-up kernel
  int bexp;         // the iteration solves A x' = 2^bexp b; the answer is x = 2^-bexp x'
  double rho_prev;  // r.z of the previous iteration (Fletcher-Reeves beta)
  // error estimate: in CG, ||x* - x_k||_A^2 = sum_{j >= k} alpha_j rho_j, so the terms of the last
  // kErrDelay iterations over the sum of all terms estimate the relative A-norm error of the
  // iterate kErrDelay steps before the end (an upper estimate for the returned one)
  double aro_total;
  double aro_ring[8];
  int aro_n;
};
constexpr int kErrDelay = 8;

// Static description of one slot (device copy).  Padded transform dims are multiples of kPad.
struct SlotDesc {
  int nx, ny, nxp, nyp;
  int bcx, bcy;
  int n_st_tiles;    // grid tiles of the set-up, residual and slicing kernels: ceil(nx/64) * ceil(ny/32)
  int n_sten_tiles;  // tiles of the stencil kernel: ceil(nx/64) * ceil(ny/sten_ty)
  int sten_ty;       // the stencil kernel's tile height (16 or 32)
  int n_vec_items;   // vector chunks: ceil(nx*ny / kVecChunk)
  int n_gm_tiles;    // output tiles of one transform stage
  float wc, wex, wey, wd, wfx, wfy;  // stencil weights (hi), scaled so that max(a, c) = 1
  float wc_l, wex_l, wey_l, wd_l, wfx_l, wfy_l;  // low parts (anisotropic grids only)
  double dwc, dwex, dwey, dwd, dwfx, dwfy;       // FP64 weights for the true residual
  int aniso;
  // grid vectors [ny][nx].  Every CG vector is a double-float pair v = hi + lo of FP32 planes
  // (about 48 bits), updated with error-free FP32 transformations: with FP32 storage alone the
  // rounding of any one of r, p, q, z costs this operator 60-100% more iterations.
  uint8_t* mask;     // 1 = unknown node
  double* b;
  float* xhi;        // the iterate x = xhi + xlo
  float* xlo;
  float* r;          // hi planes ...
  float* p[2];
  float* q;
  float* z;
  float* r_lo;       // ... and their lo planes
  float* p_lo[2];
  float* q_lo;
  float* z_lo;
  // transform intermediates of the CUDA-core path, padded [.][.] row-major, double-float planes
  float* t1;         // [nxp][nyp]
  float* t2;         // [nyp][nxp]
  float* t3;         // [nxp][nyp]
  float* t1_lo;
  float* t2_lo;
  float* t3_lo;
  const float* qx;   // [nxp][nxp]  Qx[x][k] (hi); the lo plane follows at + nxp * nxp
  const float* qxt;  // [nxp][nxp]  Qx^T
  const float* qy;
  const float* qyt;
  const float* lamx; // [nxp] eigenvalues of T_x (scaled), padding entries never read
  const float* lamy;
  float wnorm;       // 1 / w_max, so that the scaled weights are <= 1
  int zero_mode;     // 1: drop the (0,0) mode (both axes symmetric/periodic)
  // tensor-core path: block-scaled integer slices (NS 16-bit planes) and their TMA descriptors
  void* tc_r;        // [NS][nyp][nxp]  residual
  void* tc_t1;       // [NS][nxp][nyp]
  void* tc_t2;       // [NS][nyp][nxp]
  void* tc_t3;       // [NS][nxp][nyp]
  int8_t* tc_e[4];   // block exponents of the A operand of stage s: [rows][K/128]
  const int8_t* tc_eb[4];  // block exponents of the B operand of stage s (transform matrices)
  const void* tmaps; // 8 CUtensorMap (64-byte aligned): A operand of stages 0..3, B of 0..3
  const void* st_maps;  // kStMaps CUtensorMap for the stencil's tensor copies (z, z_lo, p[0],
                        // p_lo[0], p[1], p_lo[1], mask); null when a mask row is not a multiple
                        // of 16 bytes
  int n_tc_tiles;    // output tiles of one tensor-core transform stage
  // Low-mode correction of the tensor-core preconditioner: the modes kx < lowm_x, ky < lowm_y
  // (the smoothest, with the largest weights) are left out of the four 32-bit transform stages and
  // added from thin transforms with six slices per operand (about 48 bits).  0 = off.
  int lowm_x, lowm_y;
  float* low_gp;            // per forward tile t its share of G = Qy_low^T (r Qx_low): [t][2][32][32]
                            // (hi plane, then lo plane)
  void* low_jt;             // J^T slices [kLowNS][nxp][kLowK3] (16-bit codes), J = W o G Qx_low^T
  int8_t* low_jt_e;         // block exponent of each J^T row [nxp]
  float* low_z;             // zl = Qy_low J: [ny][nx] hi plane, lo plane at + nx * ny
  const float* low_qxd;     // Qx[x][kx < 32] double-float: [nxp][32] hi, lo plane at + nxp * 32
  const float* low_qyd;     // Qy[y][ky < 32] double-float: [nyp][32] hi, lo plane at + nyp * 32
  const int8_t* low_qxt_e;  // exponents of the forward product's B operand: [32][nxp / 128]
  const int8_t* low_qy_e;   // exponents of the inverse product's B operand: [nyp]
  const void* low_maps;     // 4 CUtensorMap: r slices, Qx_low^T slices, J^T slices, Qy_low slices
  int n_l1_tiles;           // tiles of the forward product: nyp / 128
  int n_l3_tiles;           // items of the inverse product: nxp / 128 (each walks every y-tile)
  // Mirror fold of the tensor-core transforms (i -> n-1-i on an axis; even and odd classes of
  // ceil(n/2) nodes each): a slot with a folded axis runs its four stages as two or four
  // half-size problems, the slot's classes, held in the tensor-core problem list at
  // kMirClasses * slot + c, c = 2 cls_y + cls_x.
  int mir;           // slot: bit 0 = x folded, bit 1 = y folded (0: the slot is its own problem)
  int mhx, mhy;      // slot: class nodes along x, y (ceil(n/2) on a folded axis, else n)
  int n_fold_items;  // slot: items of the fold kernel (8 class rows x 128 columns)
  int n_prep_items;  // slot with no folded axis: items of its residual slicing (32 rows x 128)
  int n_unfold_tiles;// slot: tiles of the unfold kernel (32 x 8 class nodes)
  int n_prec_parts;  // slot: r.z, z.q partials the preconditioner leaves (stage-3 or unfold tiles)
  int mir_out;       // class problem: stage 3 writes the class result g to z, z_lo ([ny][nx])
  SlotScalars* sc;
  double* part;      // per-work-item partial sums (2 doubles per item), slot-local indexing
  double* pq_part;   // p.q partial sums of the stencil, one per 64 x 16 block [ny/16][nx/64]
};

constexpr int kMirClasses = 4;  // tensor-core problem entries per slot

struct WorkItem {
  int slot;
  int tile;   // tile / chunk index within the slot
};

// ------------------------------------------------------------------------------------------
// Reductions
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of up to two values; result valid in thread 0.  `sh` holds >= 2*32 doubles.
template <int NT>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[w] = a; sh[32 + w] = b; }
  __syncthreads();
  if (w == 0) {
    a = (l < NT / 32) ? sh[l] : 0.0;
    b = (l < NT / 32) ? sh[32 + l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
}

// Last-item protocol, called by every thread of the block after thread 0 has written the item's
// partials.  Returns true in all threads of the item that completes the slot.
__device__ __forceinline__ bool last_item_block(unsigned* counter, unsigned total, int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    const int last = (prev == total - 1) ? 1 : 0;
    if (last) {
      __threadfence();
      *counter = 0u;
    }
    *sflag = last;
  }
  __syncthreads();
  return *sflag != 0;
}

// Sums of partials part[t*4 + k] (k = 0..K-1) over t < n, by the whole block: thread i adds
// t = i, i + NT, ... in order, then a fixed tree.  The order depends only on n, so the result is
// the same whichever block runs the reduction.  Results valid in thread 0.
template <int NT, int K>
__device__ __forceinline__ void reduce_partials(const double* part, int n, double (&out)[K],
                                                double* sh) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < n; t += NT) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(&part[t * 4 + k]);
  }
  double a = acc[0], b = K > 1 ? acc[1] : 0.0;
  block_sum2<NT>(a, b, sh);
  out[0] = a;
  if (K > 1) out[1] = b;
  if (K > 2) {
    double c = acc[2], d = 0.0;
    block_sum2<NT>(c, d, sh);
    out[2] = c;
  }
}

// ------------------------------------------------------------------------------------------
// Error-free transformations in FP32 (Knuth TwoSum, FMA-based TwoProd).  The _rn intrinsics
// are never contracted into FMAs, which keeps the transformations exact.
// ------------------------------------------------------------------------------------------
struct f2 { float hi, lo; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated accumulator (Ogita-Rump-Oishi Sum2): s + c carries about twice FP32 precision.
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float e;
    two_sum(s, x, s, e);
    c = __fadd_rn(c, e);
  }
  // add w*x for an FP32 weight w (exact product split by FMA)
  __device__ __forceinline__ void add_prod(float w, float x) {
    const float p = __fmul_rn(w, x);
    const float pe = __fmaf_rn(w, x, -p);
    add(p);
    c = __fadd_rn(c, pe);
  }
  __device__ __forceinline__ float result() const { return __fadd_rn(s, c); }
};

// Packed FP32x2 arithmetic (two independent lanes, each rounded exactly as its scalar
// counterpart): a - b is fma(b, -1, a), one rounding.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 mul2(float w, float2 a) { return __fmul2_rn(make_float2(w, w), a); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// CompSum on two lanes at once (the same operations, in the same order, per lane).
struct CompSum2 {
  float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 x) {
    float2 e;
    two_sum2(s, x, s, e);
    c = add2(c, e);
  }
  __device__ __forceinline__ float2 result() const { return add2(s, c); }
};

// Compensated FP32 dot-product accumulator (TwoProd + TwoSum per term).  GB300 runs FP64 at a
// small fraction of its FP32 rate, so per-element FP64 arithmetic would dominate the
// bandwidth-bound kernels; a thread's terms are summed here and only the per-thread totals are
// combined in FP64.
struct CompDot {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    float e;
    two_sum(s, p, s, e);
    c = __fadd_rn(c, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Block sum of compensated per-thread accumulators: FP32 TwoSum reductions inside each warp,
// FP64 only across the block's warps (thread 0).  Result valid in thread 0.  `sh` >= 32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum_comp(CompDot d, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, d.s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, d.c, o);
    float e;
    two_sum(d.s, s2, d.s, e);
    d.c = __fadd_rn(d.c, __fadd_rn(c2, e));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = d.value();
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < NT / 32; ++k) t += sh[k];
  return t;
}

// ------------------------------------------------------------------------------------------
// Double-float arithmetic (Dekker, Knuth): a value is an unevaluated FP32 pair hi + lo with
// |lo| <= ulp(hi) / 2.  Sums use TwoSum, products the FMA-based TwoProd; cross terms of size
// 2^-24 relative are added in plain FP32, so results carry about 48 bits.
// ------------------------------------------------------------------------------------------
// (s, e) -> normalised pair, valid when |e| is at most about ulp(s) (Fast2Sum)
__device__ __forceinline__ f2 df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
// a * b for a double-float a and an FP32 b
__device__ __forceinline__ f2 df_mul(f2 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_norm(p, e);
}
// a * b for double-float a and b
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}
// c + a * b, all double-float (one TwoProd, one TwoSum)
__device__ __forceinline__ f2 df_fma(f2 a, f2 b, f2 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, e;
  two_sum(c.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(c.lo, pe));
  return df_norm(s, e);
}
__device__ __forceinline__ f2 df_neg(f2 a) { return f2{-a.hi, -a.lo}; }
// an FP64 value as a double-float pair (host and device)
__host__ __device__ __forceinline__ f2 df_of(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

// Packed FP32x2 forms of the same operations (two independent lanes, each rounded exactly as its
// scalar counterpart).
struct f2x2 { float2 hi, lo; };
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2x2 df_norm2(float2 s, float2 e) {
  const float2 h = add2(s, e);
  return {h, sub2(e, sub2(h, s))};
}
// z + beta * p for double-float z, p (two lanes) and a double-float scalar beta
__device__ __forceinline__ f2x2 df_axpy2(f2 beta, f2x2 p, f2x2 z) {
  const float2 bh = make_float2(beta.hi, beta.hi), bl = make_float2(beta.lo, beta.lo);
  const float2 t = __fmul2_rn(bh, p.hi);
  float2 te = fma2(bh, p.hi, neg2(t));
  te = fma2(bh, p.lo, te);
  te = fma2(bl, p.hi, te);
  float2 s, e;
  two_sum2(z.hi, t, s, e);
  e = add2(e, add2(z.lo, te));
  return df_norm2(s, e);
}

// x += a * p with double-float x, p and scalar a (TwoProd + TwoSum)
__device__ __forceinline__ void df_axpy(float& xh, float& xl, f2 a, float ph, float pl) {
  const f2 r = df_fma(a, f2{ph, pl}, f2{xh, xl});
  xh = r.hi;
  xl = r.lo;
}

// Compensated dot product of double-float vectors: hi * hi by TwoProd into a Sum2 accumulator,
// the two cross terms (2^-24 relative) in plain FP32.
struct CompDotDF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float pe = __fmaf_rn(ah, bh, -p);
    float e;
    two_sum(s, p, s, e);
    c = __fadd_rn(c, __fadd_rn(e, __fmaf_rn(ah, bl, __fmaf_rn(al, bh, pe))));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
  __device__ __forceinline__ CompDot as_comp() const {
    CompDot d;
    d.s = s;
    d.c = c;
    return d;
  }
};
// CompDotDF on two lanes at once (the same operations, in the same order, per lane).
struct CompDotDF2 {
  float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 ah, float2 al, float2 bh, float2 bl) {
    const float2 p = __fmul2_rn(ah, bh);
    const float2 pe = __ffma2_rn(ah, bh, make_float2(-p.x, -p.y));
    float2 e;
    two_sum2(s, p, s, e);
    c = add2(c, add2(e, __ffma2_rn(ah, bl, __ffma2_rn(al, bh, pe))));
  }
};

// ------------------------------------------------------------------------------------------
// Ghost-node maps of one axis (Algorithm 1 padding; symmetric = half-sample reflection;
// periodic = wrap).  Input index i in [-2, n+1].  Returns the node index and a sign
// (+1, -1, or 0 for the zero Dirichlet boundary node).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int ghost(int i, int n, int bc, float& sgn) {
  sgn = 1.f;
  if (i >= 0 && i < n) return i;
  if (bc == BC_PER) return i < 0 ? i + n : i - n;
  if (bc == BC_SYM) return i < 0 ? -1 - i : 2 * n - 1 - i;
  // Dirichlet: distance 1 is the boundary node (zero), distance 2 the negated first node
  if (i == -1 || i == n) { sgn = 0.f; return 0; }
  sgn = -1.f;
  return i < 0 ? -i - 2 : 2 * n - i;
}

// wnorm / s^2 by the approximate division (at most 2 ulp for s^2 in [2^-126, 2^126]; s^2 of the
// grids' eigenvalue sums stays far inside that range).  The preconditioner is only an
// approximation of the inverse, so a 2-ulp change of its weights is immaterial.
__device__ __forceinline__ float spectral_weight_of(float wnorm, float s) {
  return __fdividef(wnorm, s * s);
}

// Spectral weight 1/(lam_y + lam_x)^2, normalised to <= 1; zero for padding and the constant
// mode when both axes are symmetric/periodic (pseudo-inverse).
__device__ __forceinline__ float spectral_weight(const SlotDesc& S, int kx, int ky) {
  if (kx >= S.nx || ky >= S.ny) return 0.f;
  const float s = S.lamy[ky] + S.lamx[kx];
  if (!(s > 0.f)) return 0.f;
  return spectral_weight_of(S.wnorm, s);
}

// Last item of stage 3 (thread 0): r.z, z.q -> rho, beta (flexible or Fletcher-Reeves).
__device__ __forceinline__ void finish_preconditioner(const SlotDesc& S, double rz, double zq,
                                                      int mode) {
  SlotScalars* sc = S.sc;
  if (mode == 2) {
    sc->rho = rz;
    sc->zq = zq;
    return;
  }
  // Mode 1 recomputes, after a residual replacement, the beta of the iteration whose mode-0
  // pass already ran: its Fletcher-Reeves denominator is the r.z from before that pass.
  if (mode == 0) sc->rho_prev = sc->rho;
  double beta = 0.0;
  if (sc->it > 0) beta = sc->flexible ? -zq / sc->pq : rz / sc->rho_prev;
  sc->rho = rz;
  sc->zq = zq;
  sc->beta = beta;
  if (!isfinite(rz) || !isfinite(beta)) {
    sc->status = ST_EBREAKDOWN;
    sc->active = 0;
    sc->fold = 1;
  }
  if (mode == 1) sc->need_prec = 0;
}

}  // namespace bx
