// Three-dimensional extension (Sec. 3 Example 2: the equations of Sec. 2 on an nz x ny x nx box).
//
// The operator is A = R (L_z (+) L_y (+) L_x)^2 R^T, L_a the 1-D second difference of axis a under
// its boundary rule; at an interior node with equal spacings it is the 25-point squared 7-point
// Laplacian.  It is applied as Algorithm 1 does in two dimensions, the Laplacian twice with the
// ghost rule of each axis (both passes need only the ghosts at distance one, and the boundary
// rules make the once-padded Laplacian at a ghost node the reflected, wrapped or zero one).  The
// CG vectors are double-float pairs (hi, lo) of FP32 planes as in the two-dimensional path; each
// Laplacian pass adds the seven products of the hi plane by an error-free TwoProd/TwoSum chain and
// the lo plane's in plain FP32.  The right-hand side and the residual replacements are FP64.
//
// The preconditioner is the fast Poisson solve on the box, (L^2)^+ by separable transforms along
// the three axes (Example 2: Fourier transforms on every axis; the cosine and sine transforms of
// the other rules likewise): six dense transform products with double-float operands accumulated
// by compensated dot products, each contracting the contiguous axis and writing its result with
// that axis moved to the front, so that three products rotate the box through all three axes;
// the eigenvalue weights come between the forward and the inverse three.
//
// The iteration is preconditioned CG from x = 0 with the Fletcher-Reeves beta, driven from the
// host (one scalar read per reduction); every reduction sums per-block partials in a fixed
// order, so results are reproducible bit for bit.
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace bx {
namespace {

struct Grid3 {
  int nx, ny, nz;
  int bcx, bcy, bcz;
  float cx, cy, cz;     // 1/h^2 of each axis over the largest of the three (<= 1)
  double dcx, dcy, dcz;
};

constexpr int kT = 256;  // threads of the grid kernels (32 x 8)

__device__ __forceinline__ size_t node3(const Grid3& G, int x, int y, int z) {
  return (static_cast<size_t>(z) * G.ny + y) * G.nx + x;
}

// Block sum of a double per thread in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kT / 32; ++k) s += sh[k];
  return s;
}

__device__ __forceinline__ int block_linear() {
  return (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
}

// The seven taps of the Laplacian at (x, y, z): node indices and ghost signs (0 = the Dirichlet
// boundary node, whose value is zero).
struct Taps7 {
  size_t g[7];
  float s[7];
  float w[7];
};
__device__ __forceinline__ Taps7 taps7(const Grid3& G, int x, int y, int z) {
  Taps7 t;
  float sg;
  int i;
  t.g[0] = node3(G, x, y, z);
  t.s[0] = 1.f;
  t.w[0] = 2.f * (G.cx + G.cy + G.cz);
  i = ghost(x - 1, G.nx, G.bcx, sg); t.g[1] = node3(G, i, y, z); t.s[1] = sg; t.w[1] = -G.cx;
  i = ghost(x + 1, G.nx, G.bcx, sg); t.g[2] = node3(G, i, y, z); t.s[2] = sg; t.w[2] = -G.cx;
  i = ghost(y - 1, G.ny, G.bcy, sg); t.g[3] = node3(G, x, i, z); t.s[3] = sg; t.w[3] = -G.cy;
  i = ghost(y + 1, G.ny, G.bcy, sg); t.g[4] = node3(G, x, i, z); t.s[4] = sg; t.w[4] = -G.cy;
  i = ghost(z - 1, G.nz, G.bcz, sg); t.g[5] = node3(G, x, y, i); t.s[5] = sg; t.w[5] = -G.cz;
  i = ghost(z + 1, G.nz, G.bcz, sg); t.g[6] = node3(G, x, y, i); t.s[6] = sg; t.w[6] = -G.cz;
  return t;
}

// Double-float Laplacian pass, marching along z.  A block of 32 x 8 threads owns 32 x kBy nodes of
// (x, y) (two rows per thread, ty and ty + 8) and a chunk of kZc planes.  Each thread keeps its
// own two columns in registers (planes z - 1, z, z + 1 and the two in flight); the x and y
// neighbours come from a shared-memory tile of the plane with its one-node halo, written once per
// plane and double-buffered, so one barrier per plane suffices.  Global loads run two planes ahead
// of their use.  Every cell's ghost map in x and y is taken once per thread, the z map once per
// plane; ghost signs are folded into the loaded values.  FINAL = false: out = L in at every node.
// FINAL = true: out = M L in (zero at known nodes), and the block's partial p.out (compensated).
// The terms are added in the order centre, x-1, x+1, y-1, y+1, z-1, z+1, as the single-node form
// would.
constexpr int kZc = 16;                       // planes per block
constexpr int kBy = 16;                       // rows per block
constexpr int kTw = 34, kTh = kBy + 2;        // tile with halo
constexpr int kHalo = 2 * kTw + 2 * kBy;      // halo cells of a tile
static_assert(kHalo <= kT && kBy == 2 * (kT / 32), "one halo cell per thread, two rows per thread");

// One cell that a thread loads on every plane: its offset within a plane and the product of its
// x and y ghost signs; ok = false for cells that are no node's neighbour (nothing is loaded).
struct Cell3 {
  size_t off = 0;
  float sxy = 0.f;
  bool ok = false;
};
__device__ __forceinline__ Cell3 cell3(const Grid3& G, int gx, int gy) {
  Cell3 c;
  if (gx > G.nx || gy > G.ny) return c;  // farther cells neighbour no node of the grid
  float sx, sy;
  const int mx = ghost(gx, G.nx, G.bcx, sx), my = ghost(gy, G.ny, G.bcy, sy);
  c.sxy = sx * sy;
  c.ok = c.sxy != 0.f;
  c.off = static_cast<size_t>(my) * G.nx + mx;
  return c;
}

// Tile coordinates of halo cell k: the row above, the row below, the left and the right column.
__device__ __forceinline__ int halo_pos(int k) {
  if (k < kTw) return k;
  if (k < 2 * kTw) return (kTh - 1) * kTw + (k - kTw);
  if (k < 2 * kTw + kBy) return (1 + k - 2 * kTw) * kTw;
  return (1 + k - 2 * kTw - kBy) * kTw + kTw - 1;
}

// A thread's values of one plane: its two own cells and its halo cell (hi, lo).
struct Plane3 {
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
};
__device__ __forceinline__ Plane3 k3_fetch(const Grid3& G, const float* __restrict__ ih,
                                           const float* __restrict__ il, const Cell3 (&cl)[3], int zz) {
  Plane3 p;
  float sz;
  const int mz = ghost(zz, G.nz, G.bcz, sz);
  if (sz == 0.f) return p;
  const size_t base = static_cast<size_t>(mz) * G.ny * G.nx;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (cl[k].ok) {
      const float s = cl[k].sxy * sz;
      p.h[k] = s * ih[base + cl[k].off];
      p.l[k] = s * il[base + cl[k].off];
    }
  return p;
}

__device__ __forceinline__ void k3_put(const Plane3& p, float* th, float* tl, int ca, int hp) {
  th[ca] = p.h[0];
  tl[ca] = p.l[0];
  th[ca + 8 * kTw] = p.h[1];
  tl[ca + 8 * kTw] = p.l[1];
  if (hp >= 0) {
    th[hp] = p.h[2];
    tl[hp] = p.l[2];
  }
}

// The seven-term double-float Laplacian of one node: x and y neighbours from the tile at c, the
// centre and the z neighbours (below, up) from the thread's registers.
__device__ __forceinline__ f2 k3_node(const Grid3& G, const float* th, const float* tl, int c, float ch,
                                      float cl, float bh, float bl, float uh, float ul) {
  const float w0 = 2.f * (G.cx + G.cy + G.cz);
  const float hv[7] = {ch, th[c - 1], th[c + 1], th[c - kTw], th[c + kTw], bh, uh};
  const float lv[7] = {cl, tl[c - 1], tl[c + 1], tl[c - kTw], tl[c + kTw], bl, ul};
  const float w[7] = {w0, -G.cx, -G.cx, -G.cy, -G.cy, -G.cz, -G.cz};
  CompSum a;
  float lo = 0.f;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    a.add_prod(w[k], hv[k]);
    lo = __fmaf_rn(w[k], lv[k], lo);
  }
  return df_norm(a.s, __fadd_rn(a.c, lo));
}

template <bool FINAL>
__global__ void __launch_bounds__(kT)
k3_lap(Grid3 G, const float* __restrict__ ih, const float* __restrict__ il, float* __restrict__ oh,
       float* __restrict__ ol, const uint8_t* __restrict__ mask, const float* __restrict__ ph,
       const float* __restrict__ pl, double* __restrict__ part) {
  __shared__ double sh[kT / 32];
  __shared__ float tile[2][2][kTh * kTw];  // [buffer][hi, lo]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * kBy, z0 = blockIdx.z * kZc;
  const int z1 = min(z0 + kZc, G.nz);
  const int x = x0 + tx;
  const int yr[2] = {y0 + ty, y0 + ty + 8};
  const bool in[2] = {x < G.nx && yr[0] < G.ny, x < G.nx && yr[1] < G.ny};
  const int ca = (ty + 1) * kTw + tx + 1;  // tile position of the first own node
  Cell3 cl[3];
  cl[0] = cell3(G, x, yr[0]);
  cl[1] = cell3(G, x, yr[1]);
  int hp = -1;
  if (threadIdx.x < kHalo) {
    hp = halo_pos(threadIdx.x);
    const int ly = hp / kTw, lx = hp - ly * kTw;
    cl[2] = cell3(G, x0 - 1 + lx, y0 - 1 + ly);
  }
  const size_t plane = static_cast<size_t>(G.ny) * G.nx;
  // p and the mask at the own nodes, loaded one plane ahead (FINAL only)
  uint8_t mk[2] = {0, 0};
  float pph[2] = {0.f, 0.f}, ppl[2] = {0.f, 0.f};
  auto load_p = [&](int z, uint8_t (&m)[2], float (&h)[2], float (&l)[2]) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (in[i]) {
        const size_t g = z * plane + cl[i].off;
        m[i] = mask[g];
        h[i] = ph[g];
        l[i] = pl[g];
      }
  };
  Plane3 below = k3_fetch(G, ih, il, cl, z0 - 1);
  Plane3 cur = k3_fetch(G, ih, il, cl, z0);
  Plane3 up = k3_fetch(G, ih, il, cl, z0 + 1);
  Plane3 n1;
  if (z0 + 1 < z1) n1 = k3_fetch(G, ih, il, cl, z0 + 2);
  if (FINAL) load_p(z0, mk, pph, ppl);
  k3_put(cur, tile[0][0], tile[0][1], ca, hp);
  __syncthreads();
  CompDotDF dot;
  for (int z = z0; z < z1; ++z) {
    const int b = (z - z0) & 1;
    Plane3 n2;  // plane z + 3, needed from the step of plane z + 2 on
    if (z + 2 < z1) n2 = k3_fetch(G, ih, il, cl, z + 3);
    uint8_t nmk[2] = {0, 0};
    float nph[2] = {0.f, 0.f}, npl[2] = {0.f, 0.f};
    if (FINAL && z + 1 < z1) load_p(z + 1, nmk, nph, npl);
    const float* th = tile[b][0];
    const float* tl = tile[b][1];
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (in[i]) {
        const size_t g = z * plane + cl[i].off;
        f2 v{0.f, 0.f};
        if (!FINAL || mk[i])
          v = k3_node(G, th, tl, ca + i * 8 * kTw, cur.h[i], cur.l[i], below.h[i], below.l[i], up.h[i], up.l[i]);
        oh[g] = v.hi;
        ol[g] = v.lo;
        if (FINAL) dot.add(pph[i], ppl[i], v.hi, v.lo);
      }
    if (z + 1 < z1) k3_put(up, tile[b ^ 1][0], tile[b ^ 1][1], ca, hp);
    __syncthreads();
    below = cur;
    cur = up;
    up = n1;
    n1 = n2;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      mk[i] = nmk[i];
      pph[i] = nph[i];
      ppl[i] = npl[i];
    }
  }
  if (FINAL) {
    const double s = block_sum_d(dot.value(), sh);
    if (threadIdx.x == 0) part[block_linear()] = s;
  }
}

// FP64 Laplacian pass.  MODE 0: out = L in.  MODE 1: out = -M L in (the right-hand side) and the
// partial ||out||^2.  MODE 2: out = b - M L in (the true residual), its partial ||out||^2, and the
// double-float copy (rh, rl) of out when rh is given.
template <int MODE>
__global__ void __launch_bounds__(kT)
k3_lap64(Grid3 G, const double* __restrict__ in, double* __restrict__ out, const uint8_t* __restrict__ mask,
         const double* __restrict__ b, double* __restrict__ part, float* __restrict__ rh, float* __restrict__ rl) {
  __shared__ double sh[kT / 32];
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int z = blockIdx.z;
  double sq = 0.0;
  if (x < G.nx && y < G.ny) {
    const Taps7 t = taps7(G, x, y, z);
    const size_t g = t.g[0];
    const double w[7] = {2.0 * (G.dcx + G.dcy + G.dcz), -G.dcx, -G.dcx, -G.dcy, -G.dcy, -G.dcz, -G.dcz};
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) v += w[k] * static_cast<double>(t.s[k]) * in[t.g[k]];
    if (MODE == 0) {
      out[g] = v;
    } else {
      const bool unk = mask[g] != 0;
      const double o = MODE == 1 ? (unk ? -v : 0.0) : (unk ? b[g] - v : 0.0);
      out[g] = o;
      sq = o * o;
      if (MODE == 2 && rh != nullptr) {
        const f2 d = df_of(o);
        rh[g] = d.hi;
        rl[g] = d.lo;
      }
    }
  }
  if (MODE != 0) {
    const double s = block_sum_d(sq, sh);
    if (threadIdx.x == 0) part[block_linear()] = s;
  }
}

// mask (1 = unknown), the known field as FP64 with zeros elsewhere, and counts: [0] unknown,
// [1] known, [2] NaN phi, [3] non-finite f at a known node.
__global__ void __launch_bounds__(kT)
k3_setup(size_t n, const float* __restrict__ phi, const float* __restrict__ f, int dir,
         uint8_t* __restrict__ mask, double* __restrict__ fk, unsigned long long* __restrict__ counts) {
  unsigned long long c[4] = {0, 0, 0, 0};
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT) {
    const float p = phi[i];
    const bool known = dir == 0 ? (p < 0.f) : (p > 0.f);
    if (p != p) ++c[2];
    const float fv = f[i];
    mask[i] = known ? 0 : 1;
    fk[i] = known ? static_cast<double>(fv) : 0.0;
    if (known) {
      ++c[1];
      if (!isfinite(fv)) ++c[3];
    } else {
      ++c[0];
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long v = c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&counts[k], v);
  }
}

// r = 2^-e b as a double-float pair, x = 0
__global__ void __launch_bounds__(kT)
k3_init(size_t n, const double* __restrict__ b, double s, float* __restrict__ rh, float* __restrict__ rl,
        float* __restrict__ xh, float* __restrict__ xl) {
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT) {
    const f2 d = df_of(b[i] * s);
    rh[i] = d.hi;
    rl[i] = d.lo;
    xh[i] = 0.f;
    xl[i] = 0.f;
  }
}

// x += alpha p, r -= alpha q (double-float), partial ||r||^2
__global__ void __launch_bounds__(kT)
k3_update(size_t n, f2 alpha, const float* __restrict__ ph, const float* __restrict__ pl,
          const float* __restrict__ qh, const float* __restrict__ ql, float* __restrict__ xh,
          float* __restrict__ xl, float* __restrict__ rh, float* __restrict__ rl, double* __restrict__ part) {
  __shared__ double sh[kT / 32];
  const f2 na{-alpha.hi, -alpha.lo};
  CompDotDF rr;
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT) {
    float a = xh[i], al = xl[i];
    df_axpy(a, al, alpha, ph[i], pl[i]);
    xh[i] = a;
    xl[i] = al;
    float r = rh[i], rlo = rl[i];
    df_axpy(r, rlo, na, qh[i], ql[i]);
    rh[i] = r;
    rl[i] = rlo;
    rr.add(r, rlo, r, rlo);
  }
  const double s = block_sum_d(rr.value(), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// p = z + beta p (double-float)
__global__ void __launch_bounds__(kT)
k3_direction(size_t n, f2 beta, const float* __restrict__ zh, const float* __restrict__ zl,
             float* __restrict__ ph, float* __restrict__ pl) {
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT) {
    const f2 v = df_fma(beta, f2{ph[i], pl[i]}, f2{zh[i], zl[i]});
    ph[i] = v.hi;
    pl[i] = v.lo;
  }
}

// the iterate as FP64 (for the true residual)
__global__ void __launch_bounds__(kT)
k3_to_double(size_t n, const float* __restrict__ h, const float* __restrict__ l, double* __restrict__ d) {
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT)
    d[i] = static_cast<double>(h[i]) + static_cast<double>(l[i]);
}

// masked copy of a float field into double-float planes (zero lo plane)
__global__ void __launch_bounds__(kT)
k3_load_masked(size_t n, const float* __restrict__ v, const uint8_t* __restrict__ mask, float* __restrict__ h,
               float* __restrict__ l) {
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT) {
    h[i] = mask[i] ? v[i] : 0.f;
    l[i] = 0.f;
  }
}

// out = f at known nodes (bit copy), 2^e x elsewhere
__global__ void __launch_bounds__(kT)
k3_output(size_t n, const float* __restrict__ xh, const float* __restrict__ xl, int e,
          const uint8_t* __restrict__ mask, const float* __restrict__ f, float* __restrict__ out) {
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT)
    out[i] = mask[i] ? static_cast<float>(ldexp(static_cast<double>(xh[i]) + static_cast<double>(xl[i]), e)) : f[i];
}

// Sum of partials in index order by one block (thread t adds t, t + 256, ...; then the block);
// entry i is part[i * stride].
__global__ void __launch_bounds__(kT)
k3_sum(const double* __restrict__ part, int n, double* __restrict__ out, int stride = 1) {
  __shared__ double sh[kT / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += kT) v += part[static_cast<size_t>(i) * stride];
  const double s = block_sum_d(v, sh);
  if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------------------------------------
// Transform products.  D[m][n] = sum_k A[m][k] B[n][k] for double-float A ([M][K], row-major, lo
// plane separate) and B (rows of length ldb, lo plane at + ldb * ldb), written with n first:
// out[n * M + m].  Tiles of 64 x 64, k in steps of 16 through shared memory; each thread keeps
// 4 x 4 compensated dot products (Ogita-Rump-Oishi Dot2 of double-float operands).
// ---------------------------------------------------------------------------------------------
constexpr int GM = 64, GN = 64, GK = 16;

__global__ void __launch_bounds__(kT)
k3_gemm(const float* __restrict__ A, const float* __restrict__ Al, int M, int K,
        const float* __restrict__ B, int ldb, int N, float* __restrict__ out, float* __restrict__ outl) {
  __shared__ float As[2][GK][GM + 1];
  __shared__ float Bs[2][GK][GN + 1];
  const float* Bl = B + static_cast<size_t>(ldb) * ldb;
  const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
  const int t = threadIdx.x, tm = t & 15, tn = t >> 4;
  CompDotDF acc[4][4];
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = t; e < GM * GK; e += kT) {
      const int mm = e / GK, kk = e - mm * GK;
      const int m = m0 + mm, k = k0 + kk;
      const bool ok = m < M && k < K;
      const size_t a = static_cast<size_t>(m) * K + k;
      As[0][kk][mm] = ok ? A[a] : 0.f;
      As[1][kk][mm] = ok ? Al[a] : 0.f;
    }
    for (int e = t; e < GN * GK; e += kT) {
      const int nn = e / GK, kk = e - nn * GK;
      const int n = n0 + nn, k = k0 + kk;
      const bool ok = n < N && k < K;
      const size_t a = static_cast<size_t>(n) * ldb + k;
      Bs[0][kk][nn] = ok ? B[a] : 0.f;
      Bs[1][kk][nn] = ok ? Bl[a] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = As[0][kk][tm + 16 * i];
        al[i] = As[1][kk][tm + 16 * i];
        bh[i] = Bs[0][kk][tn + 16 * i];
        bl[i] = Bs[1][kk][tn + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j].add(ah[i], al[i], bh[j], bl[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tm + 16 * i, n = n0 + tn + 16 * j;
      if (m < M && n < N) {
        const f2 v = df_norm(acc[i][j].s, acc[i][j].c);
        out[static_cast<size_t>(n) * M + m] = v.hi;
        outl[static_cast<size_t>(n) * M + m] = v.lo;
      }
    }
}

// Weights of the modes [kz][ky][kx]: wnorm / (lam_z + lam_y + lam_x)^2, zero for a zero sum (the
// constant mode when no axis is Dirichlet).
__global__ void __launch_bounds__(kT)
k3_weights(int nx, int ny, int nz, const float* __restrict__ lx, const float* __restrict__ ly,
           const float* __restrict__ lz, float wnorm, float* __restrict__ h, float* __restrict__ l) {
  const size_t n = static_cast<size_t>(nx) * ny * nz;
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT) {
    const int kx = static_cast<int>(i % nx);
    const int ky = static_cast<int>((i / nx) % ny);
    const int kz = static_cast<int>(i / (static_cast<size_t>(nx) * ny));
    const float s = lz[kz] + ly[ky] + lx[kx];
    f2 v{0.f, 0.f};
    if (s > 0.f) v = df_mul(f2{h[i], l[i]}, spectral_weight_of(wnorm, s));
    h[i] = v.hi;
    l[i] = v.lo;
  }
}

// z = M Z (zero at known nodes) and the block's partial r.z
__global__ void __launch_bounds__(kT)
k3_mask_dot(size_t n, const float* __restrict__ Zh, const float* __restrict__ Zl, const uint8_t* __restrict__ mask,
            const float* __restrict__ rh, const float* __restrict__ rl, float* __restrict__ zh,
            float* __restrict__ zl, double* __restrict__ part) {
  __shared__ double sh[kT / 32];
  CompDotDF d;
  for (size_t i = blockIdx.x * static_cast<size_t>(kT) + threadIdx.x; i < n; i += static_cast<size_t>(gridDim.x) * kT) {
    const bool u = mask[i] != 0;
    const float a = u ? Zh[i] : 0.f, b = u ? Zl[i] : 0.f;
    zh[i] = a;
    zl[i] = b;
    d.add(rh[i], rl[i], a, b);
  }
  const double s = block_sum_d(d.value(), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
#define BX3(call)                                                     \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) {                                          \
      *err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
      return EXT_ECUDA;                                               \
    }                                                                 \
  } while (0)

// Device state of one 3-D solve (allocated per call, freed on every return path).
struct State3 {
  size_t n = 0;
  int vec_blocks = 0;
  dim3 grid3, gridz, block3;  // gridz: the z-marching double-float passes
  int n_parts = 0, n_parts_z = 0;
  uint8_t* mask = nullptr;
  double *b = nullptr, *d0 = nullptr, *d1 = nullptr, *part = nullptr, *scal = nullptr;
  float *xh = nullptr, *xl = nullptr, *rh = nullptr, *rl = nullptr, *ph = nullptr, *pl = nullptr;
  float *qh = nullptr, *ql = nullptr, *zh = nullptr, *zl = nullptr, *uh = nullptr, *ul = nullptr;
  float *th = nullptr, *tl = nullptr, *lam = nullptr;
  unsigned long long* counts = nullptr;
  std::vector<void*> owned;
  Tc3 tc;  // the tensor-core preconditioner, when built
  ~State3() {
    for (void* p : owned) cudaFree(p);
    for (void* p : tc.owned) cudaFree(p);
  }
  template <class T>
  int take(T** p, size_t count, std::string* err) {
    void* v = nullptr;
    if (cudaMalloc(&v, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
      cudaGetLastError();
      *err = "cudaMalloc of the 3-D workspace failed";
      return EXT_ENOMEM;
    }
    owned.push_back(v);
    *p = static_cast<T*>(v);
    return EXT_OK;
  }
};

Grid3 grid_of(const Solve3Args& a) {
  Grid3 G;
  G.nx = a.nx;
  G.ny = a.ny;
  G.nz = a.nz;
  G.bcx = a.bc[0];
  G.bcy = a.bc[1];
  G.bcz = a.bc[2];
  const double c[3] = {1.0 / (a.h[0] * a.h[0]), 1.0 / (a.h[1] * a.h[1]), 1.0 / (a.h[2] * a.h[2])};
  const double m = std::max(c[0], std::max(c[1], c[2]));
  G.dcx = c[0] / m;
  G.dcy = c[1] / m;
  G.dcz = c[2] / m;
  G.cx = (float)G.dcx;
  G.cy = (float)G.dcy;
  G.cz = (float)G.dcz;
  return G;
}

int alloc_state(const Solve3Args& a, State3& s, bool solve, std::string* err) {
  s.n = (size_t)a.nx * a.ny * a.nz;
  s.block3 = dim3(kT);
  s.grid3 = dim3((a.nx + 31) / 32, (a.ny + 7) / 8, a.nz);
  s.n_parts = (int)(s.grid3.x * s.grid3.y * s.grid3.z);
  s.gridz = dim3(s.grid3.x, (a.ny + kBy - 1) / kBy, (a.nz + kZc - 1) / kZc);
  s.n_parts_z = (int)(s.gridz.x * s.gridz.y * s.gridz.z);
  s.vec_blocks = (int)std::min<size_t>((s.n + kT - 1) / kT, 4096);
  const size_t n = s.n;
  int rc = s.take(&s.mask, n, err);
  if (!rc) rc = s.take(&s.part, std::max(s.n_parts, s.vec_blocks), err);
  if (!rc) rc = s.take(&s.scal, 8, err);
  if (!rc) rc = s.take(&s.counts, 4, err);
  if (!rc) rc = s.take(&s.d0, n, err);
  if (!rc) rc = s.take(&s.zh, n, err);
  if (!rc) rc = s.take(&s.zl, n, err);
  if (!rc) rc = s.take(&s.th, n, err);
  if (!rc) rc = s.take(&s.tl, n, err);
  if (!rc) rc = s.take(&s.uh, n, err);
  if (!rc) rc = s.take(&s.ul, n, err);
  if (!rc) rc = s.take(&s.lam, (size_t)a.nx + a.ny + a.nz, err);
  if (!rc && solve) {
    rc = s.take(&s.b, n, err);
    if (!rc) rc = s.take(&s.d1, n, err);
    if (!rc) rc = s.take(&s.xh, n, err);
    if (!rc) rc = s.take(&s.xl, n, err);
    if (!rc) rc = s.take(&s.rh, n, err);
    if (!rc) rc = s.take(&s.rl, n, err);
    if (!rc) rc = s.take(&s.ph, n, err);
    if (!rc) rc = s.take(&s.pl, n, err);
    if (!rc) rc = s.take(&s.qh, n, err);
    if (!rc) rc = s.take(&s.ql, n, err);
  }
  return rc;
}

// Eigenvalues of each axis scaled like the stencil weights, and the weight normaliser wnorm =
// (smallest nonzero eigenvalue sum)^2.
int upload_eigen(const Solve3Args& a, const Grid3& G, State3& s, float* wnorm, std::string* err) {
  const double sc[3] = {G.dcx, G.dcy, G.dcz};
  const int n[3] = {a.nx, a.ny, a.nz};
  std::vector<float> all;
  double lo0[3], lo1[3];  // smallest and smallest nonzero of each axis
  for (int ax = 0; ax < 3; ++ax) {
    lo0[ax] = lo1[ax] = 1e300;
    for (int k = 0; k < n[ax]; ++k) {
      const double v = (float)(a.lam[ax][k] * sc[ax]);
      all.push_back((float)v);
      lo0[ax] = std::min(lo0[ax], v);
      if (v > 0) lo1[ax] = std::min(lo1[ax], v);
    }
  }
  double smin = lo0[0] + lo0[1] + lo0[2];
  if (!(smin > 0))
    smin = std::min(lo1[0] + lo0[1] + lo0[2], std::min(lo0[0] + lo1[1] + lo0[2], lo0[0] + lo0[1] + lo1[2]));
  *wnorm = (float)(smin * smin);
  BX3(cudaMemcpyAsync(s.lam, all.data(), 4 * all.size(), cudaMemcpyHostToDevice, a.stream));
  BX3(cudaStreamSynchronize(a.stream));  // `all` is a pageable source
  return EXT_OK;
}

// z = M (L^2)^+ M r: six transform products with the weights between (r, z double-float; the
// products alternate between (th, tl) and (uh, ul)).  r must be zero at known nodes.
void precondition(const Solve3Args& a, const State3& s, float wnorm, const float* rh, const float* rl,
                  float* zh, float* zl, bool with_dot) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  cudaStream_t st = a.stream;
  if (s.tc.on) {
    // the tensor-core path: its descriptors hold r, q, z and the mask of this solve
    const Tc3& t = s.tc;
    LaunchCfg c;
    c.slots = t.d_descs;
    c.stream = st;
    c.wait_cycles = t.wait_cycles;
    c.items = t.d_items[0];
    c.n_items = t.d_counts;
    c.grid = std::max(1, std::min(t.n_items[0], t.sm_count * 8));
    launch_prec_tc_prepare(c, 2, t.split);
    ++*a.launches;
    static const int kForm[7] = {-1, 0, 0, 1, 2, 2, 3};
    for (int k = 1; k < 7; ++k) {
      c.items = t.d_items[k];
      c.n_items = t.d_counts + k;
      c.grid = std::max(1, std::min(t.n_items[k], t.sm_count));
      launch_prec_tc(c, kForm[k], 2, t.split, t.d_err);
      ++*a.launches;
    }
    if (with_dot) {
      k3_sum<<<1, kT, 0, st>>>(t.part + 2, t.n_tiles3, s.scal + 1, 4);
      ++*a.launches;
    }
    return;
  }
  auto gemm = [&](const float* A, const float* Al, int M, int K, const float* B, int ldb, int N, float* o, float* ol) {
    const dim3 grid((M + GM - 1) / GM, (N + GN - 1) / GN);
    k3_gemm<<<grid, kT, 0, st>>>(A, Al, M, K, B, ldb, N, o, ol);
    ++*a.launches;
  };
  // forward: x, y, z (each contracts the contiguous axis and moves it to the front)
  gemm(rh, rl, nz * ny, nx, a.qt[0], a.np[0], nx, s.th, s.tl);   // [kx][z][y]
  gemm(s.th, s.tl, nx * nz, ny, a.qt[1], a.np[1], ny, s.uh, s.ul);  // [ky][kx][z]
  gemm(s.uh, s.ul, ny * nx, nz, a.qt[2], a.np[2], nz, s.th, s.tl);  // [kz][ky][kx]
  k3_weights<<<s.vec_blocks, kT, 0, st>>>(nx, ny, nz, s.lam, s.lam + nx, s.lam + nx + ny, wnorm, s.th, s.tl);
  ++*a.launches;
  // inverse: x, y, z
  gemm(s.th, s.tl, nz * ny, nx, a.q[0], a.np[0], nx, s.uh, s.ul);   // [x][kz][ky]
  gemm(s.uh, s.ul, nx * nz, ny, a.q[1], a.np[1], ny, s.th, s.tl);   // [y][x][kz]
  gemm(s.th, s.tl, ny * nx, nz, a.q[2], a.np[2], nz, s.uh, s.ul);   // [z][y][x]
  k3_mask_dot<<<s.vec_blocks, kT, 0, st>>>(s.n, s.uh, s.ul, s.mask, rh, rl, zh, zl, s.part);
  ++*a.launches;
  if (with_dot) k3_sum<<<1, kT, 0, st>>>(s.part, s.vec_blocks, s.scal + 1);
}

// q = M L^2 p (p double-float, zero at known nodes), p.q into scal[0]
void apply_operator(const Solve3Args& a, const Grid3& G, const State3& s, const float* ph, const float* pl,
                    float* qh, float* ql) {
  k3_lap<false><<<s.gridz, s.block3, 0, a.stream>>>(G, ph, pl, s.uh, s.ul, s.mask, nullptr, nullptr, nullptr);
  ++*a.launches;
  k3_lap<true><<<s.gridz, s.block3, 0, a.stream>>>(G, s.uh, s.ul, qh, ql, s.mask, ph, pl, s.part);
  ++*a.launches;
  k3_sum<<<1, kT, 0, a.stream>>>(s.part, s.n_parts_z, s.scal + 0);
  ++*a.launches;
}

int read_scalars(const Solve3Args& a, const State3& s, double* h, int count, std::string* err) {
  BX3(cudaMemcpyAsync(h, s.scal, sizeof(double) * count, cudaMemcpyDeviceToHost, a.stream));
  BX3(cudaStreamSynchronize(a.stream));
  return EXT_OK;
}

// mask and known field; validation of the data
int setup_mask(const Solve3Args& a, State3& s, const float* phi, const float* f, unsigned long long* cnt,
               std::string* err) {
  BX3(cudaMemsetAsync(s.counts, 0, 4 * sizeof(unsigned long long), a.stream));
  k3_setup<<<s.vec_blocks, kT, 0, a.stream>>>(s.n, phi, f, a.dir, s.mask, s.d0, s.counts);
  ++*a.launches;
  BX3(cudaGetLastError());
  BX3(cudaMemcpyAsync(cnt, s.counts, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, a.stream));
  BX3(cudaStreamSynchronize(a.stream));
  if (cnt[2] || cnt[3]) {
    *err = cnt[2] ? "phi holds NaN" : "f is not finite at a known node";
    return EXT_EINVAL;
  }
  return EXT_OK;
}

}  // namespace

int solve3d_run(const Solve3Args& a, const float* phi, const float* f, float* out, ext_result* res,
                std::string* err) {
  State3 s;
  int rc = alloc_state(a, s, true, err);
  if (rc) return rc;
  if (a.tc_build) {
    rc = a.tc_build(Tc3Io{s.rh, s.rl, s.qh, s.ql, s.zh, s.zl, s.mask}, s.tc);
    if (rc) return rc;
  }
  const Grid3 G = grid_of(a);
  float wnorm = 1.f;
  rc = upload_eigen(a, G, s, &wnorm, err);
  if (rc) return rc;
  unsigned long long cnt[4];
  rc = setup_mask(a, s, phi, f, cnt, err);
  if (rc) return rc;
  res->n_unknown = (int32_t)cnt[0];
  res->n_known = (int32_t)cnt[1];
  const bool has_dirichlet = a.bc[0] == 2 || a.bc[1] == 2 || a.bc[2] == 2;
  if (cnt[1] == 0 && !has_dirichlet) {
    *err = "no known node: the extension is not unique without a Dirichlet axis";
    return EXT_ENOKNOWN;
  }
  cudaStream_t st = a.stream;
  // b = -M L^2 E_K f (FP64) and ||b||^2
  k3_lap64<0><<<s.grid3, s.block3, 0, st>>>(G, s.d0, s.d1, s.mask, nullptr, nullptr, nullptr, nullptr);
  ++*a.launches;
  k3_lap64<1><<<s.grid3, s.block3, 0, st>>>(G, s.d1, s.b, s.mask, nullptr, s.part, nullptr, nullptr);
  ++*a.launches;
  k3_sum<<<1, kT, 0, st>>>(s.part, s.n_parts, s.scal + 2);
  ++*a.launches;
  double sc[4];
  rc = read_scalars(a, s, sc, 3, err);
  if (rc) return rc;
  const double bnorm = std::sqrt(sc[2]);
  res->iters = 0;
  res->relres_true = res->relres_rec = 0.0;
  res->err_est = 0.0;
  if (!(bnorm > 0.0) || cnt[0] == 0) {
    k3_init<<<s.vec_blocks, kT, 0, st>>>(s.n, s.b, 0.0, s.rh, s.rl, s.xh, s.xl);
    ++*a.launches;
    k3_output<<<s.vec_blocks, kT, 0, st>>>(s.n, s.xh, s.xl, 0, s.mask, f, out);
    ++*a.launches;
    BX3(cudaGetLastError());
    BX3(cudaStreamSynchronize(st));
    res->status = EXT_OK;
    return EXT_OK;
  }
  // the iteration runs on 2^-e b with ||2^-e b|| near 1
  int e = 0;
  std::frexp(bnorm, &e);
  const double scale = std::ldexp(1.0, -e);
  k3_init<<<s.vec_blocks, kT, 0, st>>>(s.n, s.b, scale, s.rh, s.rl, s.xh, s.xl);
  ++*a.launches;
  // the scaled right-hand side for the true residual: b <- 2^-e b (exact)
  k3_to_double<<<s.vec_blocks, kT, 0, st>>>(s.n, s.rh, s.rl, s.b);
  ++*a.launches;
  const double bn = bnorm * scale;
  const int maxit = a.maxit > 0 ? a.maxit : 10 * std::max(a.nx, std::max(a.ny, a.nz));
  precondition(a, s, wnorm, s.rh, s.rl, s.zh, s.zl, true);
  BX3(cudaMemcpyAsync(s.ph, s.zh, 4 * s.n, cudaMemcpyDeviceToDevice, st));
  BX3(cudaMemcpyAsync(s.pl, s.zl, 4 * s.n, cudaMemcpyDeviceToDevice, st));
  rc = read_scalars(a, s, sc, 2, err);
  if (rc) return rc;
  double rho = sc[1];
  double rnorm_last_repl = bn;
  int since_repl = 0;
  int it = 0;
  int status = EXT_ENOTCONV;
  double rel_rec = 1.0, aro_total = 0.0;
  std::vector<double> aro;
  auto true_residual = [&](bool replace, double* rel) -> int {
    k3_to_double<<<s.vec_blocks, kT, 0, st>>>(s.n, s.xh, s.xl, s.d0);
    ++*a.launches;
    k3_lap64<0><<<s.grid3, s.block3, 0, st>>>(G, s.d0, s.d1, s.mask, nullptr, nullptr, nullptr, nullptr);
    ++*a.launches;
    k3_lap64<2><<<s.grid3, s.block3, 0, st>>>(G, s.d1, s.d0, s.mask, s.b, s.part, replace ? s.rh : nullptr,
                                             replace ? s.rl : nullptr);
    ++*a.launches;
    k3_sum<<<1, kT, 0, st>>>(s.part, s.n_parts, s.scal + 3);
    ++*a.launches;
    double v[4];
    const int r2 = read_scalars(a, s, v, 4, err);
    if (r2) return r2;
    *rel = std::sqrt(v[3]) / bn;
    return EXT_OK;
  };
  while (it < maxit) {
    apply_operator(a, G, s, s.ph, s.pl, s.qh, s.ql);
    rc = read_scalars(a, s, sc, 1, err);
    if (rc) return rc;
    const double pq = sc[0];
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rho)) {
      status = EXT_EBREAKDOWN;
      break;
    }
    const double alpha = rho / pq;
    aro.push_back(alpha * rho);
    aro_total += alpha * rho;
    k3_update<<<s.vec_blocks, kT, 0, st>>>(s.n, df_of(alpha), s.ph, s.pl, s.qh, s.ql, s.xh, s.xl, s.rh, s.rl, s.part);
    ++*a.launches;
    k3_sum<<<1, kT, 0, st>>>(s.part, s.vec_blocks, s.scal + 2);
    ++*a.launches;
    rc = read_scalars(a, s, sc, 3, err);
    if (rc) return rc;
    ++it;
    ++since_repl;
    double rnorm = std::sqrt(sc[2]);
    rel_rec = rnorm / bn;
    bool replaced = false;
    if (rel_rec <= a.rtol) {
      // converged by the recursive residual: confirm with the FP64 true residual
      double rel = 0.0;
      rc = true_residual(true, &rel);
      if (rc) return rc;
      replaced = true;
      if (rel <= a.rtol) {
        status = EXT_OK;
        res->relres_true = rel;
        break;
      }
      rnorm = rel * bn;
    } else if (rnorm < a.replace_factor * rnorm_last_repl || since_repl >= a.true_res_every) {
      double rel = 0.0;
      rc = true_residual(true, &rel);
      if (rc) return rc;
      replaced = true;
      rnorm = rel * bn;
    }
    if (replaced) {
      rnorm_last_repl = rnorm;
      since_repl = 0;
    }
    precondition(a, s, wnorm, s.rh, s.rl, s.zh, s.zl, true);
    rc = read_scalars(a, s, sc, 2, err);
    if (rc) return rc;
    const double rho_new = sc[1];
    const double beta = rho_new / rho;
    if (!std::isfinite(beta)) {
      status = EXT_EBREAKDOWN;
      break;
    }
    rho = rho_new;
    k3_direction<<<s.vec_blocks, kT, 0, st>>>(s.n, df_of(beta), s.zh, s.zl, s.ph, s.pl);
    ++*a.launches;
  }
  if (status != EXT_OK) {
    double rel = 0.0;
    rc = true_residual(false, &rel);
    if (rc) return rc;
    res->relres_true = rel;
  }
  res->iters = it;
  res->relres_rec = rel_rec;
  double tail = 0.0;
  for (size_t k = aro.size() > 8 ? aro.size() - 8 : 0; k < aro.size(); ++k) tail += aro[k];
  res->err_est = aro_total > 0.0 ? std::sqrt(std::max(0.0, tail) / aro_total) : 0.0;
  k3_output<<<s.vec_blocks, kT, 0, st>>>(s.n, s.xh, s.xl, e, s.mask, f, out);
  ++*a.launches;
  BX3(cudaGetLastError());
  BX3(cudaStreamSynchronize(st));
  if (s.tc.on) {
    // a bounded wait of the tensor-core kernels that ran out
    int flag = 0;
    BX3(cudaMemcpy(&flag, s.tc.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      BX3(cudaMemset(s.tc.d_err, 0, sizeof(int)));
      *err = "a bounded device wait (tensor-core pipeline) ran out";
      res->status = EXT_ETIMEOUT;
      return EXT_ETIMEOUT;
    }
  }
  res->status = status;
  return status == EXT_OK ? EXT_OK : status;
}

int apply3d_operator(const Solve3Args& a, const float* phi, const float* p, float* q, std::string* err) {
  State3 s;
  int rc = alloc_state(a, s, false, err);
  if (rc) return rc;
  const Grid3 G = grid_of(a);
  unsigned long long cnt[4];
  rc = setup_mask(a, s, phi, phi, cnt, err);  // f is not used: phi stands in (finite at known nodes)
  if (rc) return rc;
  // p masked into (th, tl); q into (zh, zl); the hi plane is the result
  k3_load_masked<<<s.vec_blocks, kT, 0, a.stream>>>(s.n, p, s.mask, s.th, s.tl);
  ++*a.launches;
  apply_operator(a, G, s, s.th, s.tl, s.zh, s.zl);
  BX3(cudaMemcpyAsync(q, s.zh, 4 * s.n, cudaMemcpyDeviceToDevice, a.stream));
  BX3(cudaGetLastError());
  BX3(cudaStreamSynchronize(a.stream));
  return EXT_OK;
}

int apply3d_preconditioner(const Solve3Args& a, const float* phi, const float* r, float* z, double* scale,
                           std::string* err) {
  State3 s;
  int rc = alloc_state(a, s, false, err);
  if (rc) return rc;
  const Grid3 G = grid_of(a);
  float wnorm = 1.f;
  rc = upload_eigen(a, G, s, &wnorm, err);
  if (rc) return rc;
  unsigned long long cnt[4];
  rc = setup_mask(a, s, phi, phi, cnt, err);
  if (rc) return rc;
  // r masked into (th, tl) is consumed by the first product, so it is kept in (zh, zl)'s place:
  // the masked copy goes to d0 reinterpreted as two float planes
  float* rh = reinterpret_cast<float*>(s.d0);
  float* rl = rh + s.n;
  if (a.tc_build) {
    // z.q of the last product's epilogue is not used here: q = zeros
    BX3(cudaMemsetAsync(s.uh, 0, 4 * s.n, a.stream));
    BX3(cudaMemsetAsync(s.ul, 0, 4 * s.n, a.stream));
    rc = a.tc_build(Tc3Io{rh, rl, s.uh, s.ul, s.zh, s.zl, s.mask}, s.tc);
    if (rc) return rc;
  }
  k3_load_masked<<<s.vec_blocks, kT, 0, a.stream>>>(s.n, r, s.mask, rh, rl);
  ++*a.launches;
  precondition(a, s, wnorm, rh, rl, s.zh, s.zl, false);
  BX3(cudaMemcpyAsync(z, s.zh, 4 * s.n, cudaMemcpyDeviceToDevice, a.stream));
  BX3(cudaGetLastError());
  BX3(cudaStreamSynchronize(a.stream));
  // weights are (L^2)^+ scaled by wnorm, times the square of the stencil scaling (max 1/h^2)^-2
  const double m = std::max(1.0 / (a.h[0] * a.h[0]), std::max(1.0 / (a.h[1] * a.h[1]), 1.0 / (a.h[2] * a.h[2])));
  if (scale) *scale = (double)wnorm * m * m;
  return EXT_OK;
}

}  // namespace bx
