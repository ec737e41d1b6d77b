// C ABI of the biharmonic extension library: contexts, transform plans, solve workspaces and
// the host loop that replays CUDA-graph-captured blocks of PCG iterations.
//
// One solve (Algorithm 1): set-up kernel (mask from sign(phi), b = -M L^2 E_K f), one
// preconditioner pass, then graph replays of G iterations
//   [stencil (p = z + beta p, q = M L^2 p, p.q) -> update (x += alpha p in FP64, r, r.r) ->
//    4 transform stages (z = M (L^2)^+ M r, r.z, z.q)] x G  +  tail [FP64 true residual for slots
//    due a replacement -> 4 transform stages for slots that continue]
// until every slot reports a final status.  Batches and the serving loop use the same kernels
// over work lists that span all slots.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/biharm_ext.h"
#include "common.cuh"
#include "kernels.h"
#include "plan.h"

using namespace bx;

namespace {

thread_local std::string g_last_error;

#define BX_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      g_last_error = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return EXT_ECUDA;                                                                      \
    }                                                                                        \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct PlanDev {
  int n = 0, np = 0, bc = 0;
  int cls = -1;   // -1: the axis basis; 0 / 1: its even / odd mirror class (n = ceil(nfull / 2))
  int nfull = 0;  // nodes of the axis
  float* q = nullptr;   // [2][np][np]: hi plane, lo plane
  float* qt = nullptr;  // [2][np][np]
  std::vector<double> lam;
  void* tc = nullptr;   // tensor-core operand planes: [Q planes][Q^T planes], 2-byte elements
  int tc_split = -1;
  // low-mode operands (six slices): Q^T rows k < 32 [6][32][np] with exponents [32][np/128];
  // Q columns k < 32 as rows [6][np][64] with exponents [np]; Q[:, :32] double-float [2][np][32]
  void* low = nullptr;
  size_t low_off_te = 0, low_off_q = 0, low_off_qe = 0, low_off_d = 0;
};

// One problem's device state inside a workspace.
struct SlotHost {
  ext_problem prob{};
  SlotDesc d{};
  SlotDesc tcp[kMirClasses]{};  // tensor-core problems (mixed modes): the slot, or its classes
  int n_tcp = 0;
  char* arena = nullptr;
  size_t bytes = 0;
  float* phi_stage = nullptr;  // device copies when the caller passes host arrays
  float* f_stage = nullptr;
  float* out_stage = nullptr;
};

struct Workspace {
  std::string key;
  std::vector<SlotHost> slots;
  SlotDesc* d_slots = nullptr;
  SlotScalars* d_sc = nullptr;
  SlotScalars* h_sc = nullptr;  // pinned
  WorkItem *d_st = nullptr, *d_vec = nullptr, *d_gm = nullptr;
  WorkItem* d_sl = nullptr;     // one item per slot (tile 0), for the per-slot scalar kernels
  int *d_counts = nullptr;      // [0] grid tiles, [1] vector items, [2] gemm items, [3] slots,
                                // [4] stencil tiles, [5] [6] low-mode tiles, [7] fold items,
                                // [8] unfold tiles, [9] tensor-core problems, [10] grid tiles
                                // of unfolded slots
  int n_st = 0, n_vec = 0, n_gm = 0, n_sl = 0;
  WorkItem* d_sten = nullptr;   // the stencil kernel's tiles (64 x sten_ty)
  int n_sten = 0;
  int sten_ty = 32;             // stencil tile height of this workspace (autotuned)
  bool tuned = false;
  WorkItem *d_l1 = nullptr, *d_l3 = nullptr;  // tiles of the low-mode products
  int n_l1 = 0, n_l3 = 0;
  // tensor-core problems (mixed modes): kMirClasses entries per slot, the slot's own descriptor
  // or its mirror classes; items of the fold and unfold kernels; one item per problem
  SlotDesc* d_tcp = nullptr;
  WorkItem *d_fold = nullptr, *d_unfold = nullptr, *d_tcl = nullptr;
  int n_fold = 0, n_unfold = 0, n_tcl = 0;
  WorkItem* d_prep = nullptr;  // residual slicing of the unfolded slots (32 rows x 128 columns)
  int n_prep = 0;
  const float** d_phis = nullptr;
  const float** d_fs = nullptr;
  float** d_outs = nullptr;
  int* d_dirs = nullptr;
  void* h_ptrs = nullptr;       // pinned staging for the pointer arrays
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  int64_t graph_nodes = 0;
  void* d_tmaps = nullptr;      // per slot 8 CUtensorMap (tensor-core modes)
  struct Ev { int kind; cudaEvent_t a, b; };
  std::vector<Ev> graph_events;  // profiling: event-record nodes of the graph
  bool aniso = false;
  bool host_io = false;
  cudaStream_t stream = nullptr;  // the context's stream, or the serving worker's own
};

int plan_key(int n, int bc, int cls) { return (n * 4 + bc) * 3 + cls + 1; }

AxisBasis plan_basis(int nfull, int bc, int cls) {
  return cls < 0 ? make_axis_basis(nfull, bc) : make_class_basis(nfull, bc, cls);
}

}  // namespace

struct ext_ctx {
  int device = 0;
  int sm_count = 148;
  int cc_major = 0, cc_minor = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ext_options opt{};
  std::map<int, PlanDev> plans;
  std::map<std::string, Workspace*> ws;
  std::mutex api_mu;  // serialises ext_solve* and the serving worker on the stream
  bool tc = false;    // mixed modes: tensor-core preconditioner
  int split = 0;      // type of the exact integer operand slices: 0 = FP16, 1 = BF16
  int* d_err = nullptr;   // device flag raised by a bounded wait that ran out
  int* h_err = nullptr;   // pinned copy
  // launch accounting and optional per-kernel timing (ext_options.profile)
  std::atomic<int64_t> launches{0};
  std::recursive_mutex plan_mu;  // plan cache: shared by user threads and the serving worker
  using Pending = Workspace::Ev;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[EXT_KERNEL_KINDS] = {0};
  int64_t prof_n[EXT_KERNEL_KINDS] = {0};
  int last_tile_y = 0;  // stencil tile height of the last solve's workspace
  // serving
  struct Serve;
  Serve* serve = nullptr;
};

// ---------------------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------------------
int bx::validate_problem(const ext_problem* p) {
  if (!p) return EXT_EINVAL;
  if (p->nx < 4 || p->ny < 4) return EXT_EINVAL;
  if ((int64_t)p->nx * p->ny > (int64_t)1 << 30) return EXT_EINVAL;
  if (!(p->hx > 0.0) || !(p->hy > 0.0) || !std::isfinite(p->hx) || !std::isfinite(p->hy))
    return EXT_EINVAL;
  if (p->bc_x < 0 || p->bc_x > 2 || p->bc_y < 0 || p->bc_y > 2) return EXT_EINVAL;
  if (p->dir != 0 && p->dir != 1) return EXT_EINVAL;
  return EXT_OK;
}

bool bx::is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- tensor-core operands --------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  }
  return fn;
}

// 2-D map over `rows` rows of `inner` elements of `elem` bytes, boxes of box_inner x box_rows.
// Cells outside the array read as zeros.
static int make_tmap_2d(CUtensorMap* m, void* base, CUtensorMapDataType type, uint64_t elem, uint64_t inner,
                        uint64_t rows, uint32_t box_inner, uint32_t box_rows, CUtensorMapSwizzle swz) {
  EncodeTiledFn enc = get_encoder();
  if (!enc) {
    g_last_error = "cuTensorMapEncodeTiled not available";
    return EXT_ENOTSUP;
  }
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * elem};
  const cuuint32_t box[2] = {box_inner, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, type, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    g_last_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return EXT_ECUDA;
  }
  return EXT_OK;
}

// Tensor-core operand planes: `rows` rows of `inner` 16-bit slices; boxes of 64 x box_rows,
// 128-byte swizzle.
static int make_tmap(CUtensorMap* m, void* base, bool bf16, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  return make_tmap_2d(m, base, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                      inner, rows, 64, box_rows, CU_TENSOR_MAP_SWIZZLE_128B);
}

// Stencil windows: the hi and lo planes of z, p[0], p[1] as FP32 boxes of the tile plus its halo
// (two extra columns on the left keep each copy's start on a 16-byte boundary) and the mask as
// 8-bit boxes of the tile.  The mask rows must span a multiple of 16 bytes (nx % 16 == 0).
static bool stencil_copies_fit(int nx) { return nx % 16 == 0; }
static int make_stencil_maps(CUtensorMap (&m)[kStMaps], const SlotDesc& d, int ty) {
  const uint32_t wx = kStWinX, wy = (uint32_t)ty + 4;
  float* const vec[6] = {d.z, d.z_lo, d.p[0], d.p_lo[0], d.p[1], d.p_lo[1]};
  for (int k = 0; k < 6; ++k) {
    const int rc = make_tmap_2d(&m[k], vec[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d.nx, d.ny, wx, wy,
                                CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
  }
  return make_tmap_2d(&m[6], d.mask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d.nx, d.ny, kStTileX, (uint32_t)ty,
                      CU_TENSOR_MAP_SWIZZLE_NONE);
}

// ns integer slices of v for block exponent E (v = c0 2^(E-8) + c1 2^(E-16) + ... +
// c_{ns-1} 2^(E-8 ns)), stored as FP16 or BF16 (integers of at most 9 bits are exact in both).
static void slice_host(double v, int E, int split, int ns, uint16_t* out, size_t plane, size_t idx) {
  double r = v;
  for (int k = 0; k < ns; ++k) {
    const double c = std::nearbyint(std::ldexp(r, 8 * (k + 1) - E));
    r -= std::ldexp(c, E - 8 * (k + 1));
    out[k * plane + idx] = split == 0 ? __half_as_ushort(__double2half(c))
                                      : __bfloat16_as_ushort(__double2bfloat16(c));
  }
}

// Block exponent of `count` values: max |v| < 2^E and max |v| 2^(8-E) < 255.5 (the leading
// slice stays within +-255); 0 for an all-zero block.
static int block_exp_host(const double* v, size_t stride, int count) {
  double m = 0.0;
  for (int k = 0; k < count; ++k) m = std::max(m, std::fabs(v[k * stride]));
  if (!(m > 0.0)) return 0;
  int e;
  std::frexp(m, &e);
  if (count > 64 && std::ldexp(m, 8 - e) >= 255.5) ++e;
  return std::max(e, -90);
}

// Q and Q^T of one axis (n nodes, rule bc) as block-scaled slices, zero-padded to np x np, with
// their exponents: h = [Q slices (NS planes)][Q^T slices (NS planes)], each plane [np][np];
// ex = [exponents of Q rows][exponents of Q^T rows], each [np][np / KB].
static void slice_plan_basis(const AxisBasis& B, int np, int split, std::vector<uint16_t>& h,
                             std::vector<int8_t>& ex) {
  const int n = B.n;
  const int NS = tc_planes(split);
  const int KB = tc_block();  // k per block exponent of the sliced operands
  const int nkb = np / KB;
  const size_t plane = (size_t)np * np;
  h.assign(2 * NS * plane, 0);
  ex.assign(2 * (size_t)np * nkb, 0);
  std::vector<double> Qp((size_t)np * np, 0.0), QTp((size_t)np * np, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      Qp[(size_t)i * np + k] = B.Q[(size_t)i * n + k];
      QTp[(size_t)k * np + i] = B.Q[(size_t)i * n + k];
    }
  for (int t = 0; t < 2; ++t) {
    const std::vector<double>& M = t == 0 ? Qp : QTp;
    uint16_t* out = h.data() + t * NS * plane;
    int8_t* eo = ex.data() + t * (size_t)np * nkb;
    for (int row = 0; row < np; ++row)
      for (int kb = 0; kb < nkb; ++kb) {
        const double* blk = M.data() + (size_t)row * np + kb * KB;
        const int E = block_exp_host(blk, 1, KB);
        eo[(size_t)row * nkb + kb] = (int8_t)E;
        for (int k = 0; k < KB; ++k)
          slice_host(blk[k], E, split, NS, out, plane, (size_t)row * np + kb * KB + k);
      }
  }
}

static void slice_plan_host(int n, int bc, int np, int split, std::vector<uint16_t>& h,
                            std::vector<int8_t>& ex) {
  slice_plan_basis(make_axis_basis(n, bc), np, split, h, ex);
}

static int ensure_tc_plan(ext_ctx* ctx, PlanDev* P) {
  if (P->tc && P->tc_split == ctx->split) return EXT_OK;
  if (P->tc) {
    cudaFree(P->tc);
    P->tc = nullptr;
  }
  std::vector<uint16_t> h;
  std::vector<int8_t> ex;
  const AxisBasis B = plan_basis(P->nfull, P->bc, P->cls);
  slice_plan_basis(B, P->np, ctx->split, h, ex);
  const size_t bytes = 2 * h.size() + ex.size();
  if (cudaMalloc(&P->tc, bytes) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = "cudaMalloc of tensor-core plan failed";
    return EXT_ENOMEM;
  }
  BX_CUDA(cudaMemcpy(P->tc, h.data(), 2 * h.size(), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy((char*)P->tc + 2 * h.size(), ex.data(), ex.size(), cudaMemcpyHostToDevice));
  P->tc_split = ctx->split;
  // low-mode operands of the same basis
  if (P->low) {
    cudaFree(P->low);
    P->low = nullptr;
  }
  const int np = P->np, nkb = np / tc_block();
  const int m = std::min(kLowM, P->n);
  auto Qv = [&](int i, int k) { return (i < P->n && k < m) ? B.Q[(size_t)i * P->n + k] : 0.0; };
  const size_t pt = (size_t)kLowM * np, pq = (size_t)np * kLowK3;
  std::vector<uint16_t> lt(kLowNS * pt, 0), lq(kLowNS * pq, 0);
  std::vector<int8_t> lte((size_t)kLowM * nkb, 0), lqe(np, 0);
  std::vector<float> ld(2 * (size_t)np * kLowM, 0.f);
  std::vector<double> blk(std::max(tc_block(), kLowK3));
  for (int k = 0; k < kLowM; ++k)      // forward B operand: row k = Q[:, k], 128-wide blocks along i
    for (int kb = 0; kb < nkb; ++kb) {
      for (int t = 0; t < tc_block(); ++t) blk[t] = Qv(kb * tc_block() + t, k);
      const int E = block_exp_host(blk.data(), 1, tc_block());
      lte[(size_t)k * nkb + kb] = (int8_t)E;
      for (int t = 0; t < tc_block(); ++t)
        slice_host(blk[t], E, ctx->split, kLowNS, lt.data(), pt, (size_t)k * np + kb * tc_block() + t);
    }
  for (int i = 0; i < np; ++i) {       // inverse B operand: row i = Q[i, :32], one block
    for (int t = 0; t < kLowK3; ++t) blk[t] = t < kLowM ? Qv(i, t) : 0.0;
    const int E = block_exp_host(blk.data(), 1, kLowK3);
    lqe[i] = (int8_t)E;
    for (int t = 0; t < kLowK3; ++t) slice_host(blk[t], E, ctx->split, kLowNS, lq.data(), pq, (size_t)i * kLowK3 + t);
    for (int k = 0; k < kLowM; ++k) {
      const double v = Qv(i, k);
      const float hi = (float)v;
      ld[(size_t)i * kLowM + k] = hi;
      ld[(size_t)np * kLowM + (size_t)i * kLowM + k] = (float)(v - (double)hi);
    }
  }
  P->low_off_te = 2 * lt.size();
  P->low_off_q = align_up(P->low_off_te + lte.size(), 256);
  P->low_off_qe = P->low_off_q + 2 * lq.size();
  P->low_off_d = align_up(P->low_off_qe + lqe.size(), 256);
  const size_t lbytes = P->low_off_d + 4 * ld.size();
  if (cudaMalloc(&P->low, lbytes) != cudaSuccess) {
    cudaGetLastError();
    P->low = nullptr;
    g_last_error = "cudaMalloc of low-mode plan failed";
    return EXT_ENOMEM;
  }
  char* L = (char*)P->low;
  BX_CUDA(cudaMemcpy(L, lt.data(), 2 * lt.size(), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy(L + P->low_off_te, lte.data(), lte.size(), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy(L + P->low_off_q, lq.data(), 2 * lq.size(), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy(L + P->low_off_qe, lqe.data(), lqe.size(), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy(L + P->low_off_d, ld.data(), 4 * ld.size(), cudaMemcpyHostToDevice));
  return EXT_OK;
}

// Exponent arrays of a plan: t = 0 for Q rows, 1 for Q^T rows.
static const int8_t* plan_exps(const PlanDev* P, int t) {
  const size_t plane = (size_t)P->np * P->np;
  const size_t nkb = P->np / tc_block();
  return (const int8_t*)((const char*)P->tc + 2 * 2 * (size_t)tc_planes(P->tc_split) * plane) +
         t * (size_t)P->np * nkb;
}

static int get_plan(ext_ctx* ctx, int n, int bc, int cls, PlanDev** out) {
  const int key = plan_key(n, bc, cls);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    *out = &it->second;
    return EXT_OK;
  }
  AxisBasis B = plan_basis(n, bc, cls);
  PlanDev P;
  P.n = B.n;
  P.nfull = n;
  P.cls = cls;
  P.bc = bc;
  P.np = pad_to(B.n, kPad);
  P.lam = B.lam;
  std::vector<float> q, qt;
  padded_df(B, P.np, q, qt);
  const size_t bytes = 2 * (size_t)P.np * P.np * sizeof(float);
  if (cudaMalloc(&P.q, bytes) != cudaSuccess || cudaMalloc(&P.qt, bytes) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = "cudaMalloc of transform plan failed";
    return EXT_ENOMEM;
  }
  BX_CUDA(cudaMemcpy(P.q, q.data(), bytes, cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy(P.qt, qt.data(), bytes, cudaMemcpyHostToDevice));
  auto res = ctx->plans.emplace(key, std::move(P));
  *out = &res.first->second;
  return EXT_OK;
}

// Stencil weights of (L_y (+) L_x)^2 scaled by 1/max(a, c)^2, a = 1/hx^2, c = 1/hy^2
// (eq. discrete_biharmonic for hx = hy: 20, -8, 2, 1).
void bx::set_weights(SlotDesc& d, double hx, double hy) {
  double a = 1.0 / (hx * hx), c = 1.0 / (hy * hy);
  const double m = std::max(a, c);
  a /= m;
  c /= m;
  const double w[6] = {6 * a * a + 8 * a * c + 6 * c * c, -4 * a * a - 4 * a * c,
                       -4 * c * c - 4 * a * c, 2 * a * c, a * a, c * c};
  float* hi[6] = {&d.wc, &d.wex, &d.wey, &d.wd, &d.wfx, &d.wfy};
  float* lo[6] = {&d.wc_l, &d.wex_l, &d.wey_l, &d.wd_l, &d.wfx_l, &d.wfy_l};
  double* dw[6] = {&d.dwc, &d.dwex, &d.dwey, &d.dwd, &d.dwfx, &d.dwfy};
  for (int i = 0; i < 6; ++i) {
    *hi[i] = (float)w[i];
    *lo[i] = (float)(w[i] - (double)*hi[i]);
    *dw[i] = w[i];
  }
  d.aniso = (a != c) ? 1 : 0;
}

static void free_workspace(Workspace* W) {
  if (!W) return;
  if (W->graph) cudaGraphExecDestroy(W->graph);
  for (auto& e : W->graph_events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto& s : W->slots) cudaFree(s.arena);
  cudaFree(W->d_slots);
  cudaFree(W->d_sc);
  cudaFree(W->d_st);
  cudaFree(W->d_sten);
  cudaFree(W->d_vec);
  cudaFree(W->d_gm);
  cudaFree(W->d_sl);
  cudaFree(W->d_l1);
  cudaFree(W->d_l3);
  cudaFree(W->d_tcp);
  cudaFree(W->d_fold);
  cudaFree(W->d_unfold);
  cudaFree(W->d_tcl);
  cudaFree(W->d_prep);
  cudaFree(W->d_counts);
  cudaFree(W->d_phis);
  cudaFree(W->d_fs);
  cudaFree(W->d_outs);
  cudaFree(W->d_dirs);
  cudaFreeHost(W->h_sc);
  cudaFreeHost(W->h_ptrs);
  delete W;
}

static std::string shape_key(int count, const ext_problem* probs, bool host_io) {
  std::string k = host_io ? "H" : "D";
  char buf[160];
  for (int i = 0; i < count; ++i) {
    const ext_problem& p = probs[i];
    snprintf(buf, sizeof(buf), "|%d,%d,%d,%d,%.17g", p.nx, p.ny, p.bc_x, p.bc_y, p.hx / p.hy);
    k += buf;
  }
  return k;
}

// Device state of one problem: plans, arena layout (allocated here unless `arena` is given), slot
// descriptor, its tensor-core problems and their tensor maps.  With size_only, only s.bytes is
// computed.
static int build_slot(ext_ctx* ctx, const ext_problem& prob, bool host_io, SlotHost& s,
                      char* arena = nullptr, bool size_only = false, bool large_call = false) {
  std::lock_guard<std::recursive_mutex> plk(ctx->plan_mu);
  s.prob = prob;
  s.d = SlotDesc{};
  s.n_tcp = 0;
  const int nx = prob.nx, ny = prob.ny;
  PlanDev *px, *py;
  int rc = get_plan(ctx, nx, prob.bc_x, -1, &px);
  if (rc) return rc;
  rc = get_plan(ctx, ny, prob.bc_y, -1, &py);
  if (rc) return rc;
  SlotDesc& d = s.d;
  d.nx = nx;
  d.ny = ny;
  d.nxp = px->np;
  d.nyp = py->np;
  d.bcx = prob.bc_x;
  d.bcy = prob.bc_y;
  d.n_st_tiles = ((nx + kStTileX - 1) / kStTileX) * ((ny + kStTileY - 1) / kStTileY);
  d.sten_ty = 32;
  d.n_sten_tiles = d.n_st_tiles;
  const size_t N = (size_t)nx * ny;
  d.n_vec_items = (int)((N + kVecChunk - 1) / kVecChunk);
  const int n_gm = (d.nxp / 128) * (d.nyp / 64);
  d.n_gm_tiles = n_gm;
  d.n_tc_tiles = n_gm;
  set_weights(d, prob.hx, prob.hy);
  // the tensor-core transforms fold an axis by its mirror symmetry where both classes, padded,
  // fit in the padded axis: each stage then does half the products
  d.mir = 0;
  if (ctx->opt.fold) {
    if (mirror_pays(nx, kPad)) d.mir |= 1;
    if (mirror_pays(ny, kPad)) d.mir |= 2;
  }
  d.mhx = (d.mir & 1) ? mirror_half(nx) : nx;
  d.mhy = (d.mir & 2) ? mirror_half(ny) : ny;
  // fold items: mixed modes 8 class rows x 128 columns (a warp per row); CUDA cores 32 x 8 class
  // nodes (one per thread, the unfold tiles)
  d.n_fold_items = !d.mir ? 0 : ctx->tc ? ((d.mhy + 7) / 8) * ((d.mhx + 127) / 128) : 0;
  d.n_prep_items = (ctx->tc && !d.mir) ? ((ny + kStTileY - 1) / kStTileY) * ((nx + 127) / 128) : 0;
  d.n_unfold_tiles = d.mir ? ((d.mhx + 31) / 32) * ((d.mhy + 7) / 8) : 0;
  d.n_prec_parts = d.mir ? d.n_unfold_tiles : n_gm;
  const int n_part = std::max(std::max(d.n_st_tiles, d.n_vec_items), std::max(n_gm, d.n_unfold_tiles));
  const size_t Np = (size_t)d.nxp * d.nyp;
  // arena layout
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_b = take(8 * N), o_x = take(4 * N), o_xl = take(4 * N);
  const size_t o_part = take(8 * 4 * (size_t)n_part);
  const size_t o_pqp = take(8 * (size_t)((ny + 15) / 16) * ((nx + 31) / 32));
  const size_t o_r = take(4 * N), o_p0 = take(4 * N), o_p1 = take(4 * N);
  const size_t o_q = take(4 * N), o_z = take(4 * N), o_mask = take(N);
  const size_t o_rl = take(4 * N), o_p0l = take(4 * N), o_p1l = take(4 * N);
  const size_t o_ql = take(4 * N), o_zl = take(4 * N);
  // CUDA-core transform intermediates (hi, lo planes) of an unfolded slot
  const size_t fp = (ctx->tc || d.mir) ? 0 : 4 * Np;
  const size_t o_t1 = take(fp), o_t2 = take(fp), o_t3 = take(fp);
  const size_t o_t1l = take(fp), o_t2l = take(fp), o_t3l = take(fp);
  const size_t o_lx = take(4 * (size_t)d.nxp), o_ly = take(4 * (size_t)d.nyp);
  size_t o_io = 0;
  if (host_io) o_io = take(12 * N);
  const bool st_copy = stencil_copies_fit(nx);
  const size_t o_smaps = st_copy ? take(kStMaps * sizeof(CUtensorMap)) : 0;
  // tensor-core problems: the slot itself, or its classes c = 2 cls_y + cls_x
  struct TcLay {
    int c = 0;
    PlanDev *px = nullptr, *py = nullptr;
    size_t o_tr = 0, o_tt1 = 0, o_tt2 = 0, o_tt3 = 0, o_maps = 0, o_ex = 0, o_lx = 0, o_ly = 0;
    size_t o_g = 0, o_lh = 0, o_ljt = 0, o_ljte = 0, o_lz = 0, o_lmaps = 0;
    size_t o_s1 = 0, o_s2 = 0, o_s3 = 0, o_cr = 0;  // CUDA-core class problems: T1..T3, residual
  };
  std::vector<TcLay> tl;
  const int NS = ctx->tc ? tc_planes(ctx->split) : 0;
  // the low-mode correction: always (1), never (0), or (2) for grids of side >= 2048 and for every
  // grid of a call whose grids hold >= 2048^2 nodes together (large_call): there the correction's
  // kernels run at throughput and the iterations they save outweigh their cost; on one smaller
  // grid they are latency-bound and cost more than they save
  const bool low = ctx->tc && (ctx->opt.low_modes == 1 ||
                               (ctx->opt.low_modes == 2 &&
                                (std::max(nx, ny) >= kLowAutoSide || large_call)));
  // transform problems: in mixed modes always (the slot itself or its classes), on the CUDA
  // cores only for a folded slot (its classes; an unfolded slot runs on its own buffers)
  if (ctx->tc || d.mir) {
    for (int cy = 0; cy < ((d.mir & 2) ? 2 : 1); ++cy)
      for (int cx = 0; cx < ((d.mir & 1) ? 2 : 1); ++cx) {
        TcLay L;
        L.c = 2 * cy + cx;
        rc = get_plan(ctx, nx, prob.bc_x, (d.mir & 1) ? cx : -1, &L.px);
        if (!rc) rc = get_plan(ctx, ny, prob.bc_y, (d.mir & 2) ? cy : -1, &L.py);
        if (rc) return rc;
        const size_t Npc = (size_t)L.px->np * L.py->np;
        if (ctx->tc) {
          L.o_tr = take(2 * (low ? kLowNS : NS) * Npc);
          L.o_tt1 = take(2 * NS * Npc);
          L.o_tt2 = take(2 * NS * Npc);
          L.o_tt3 = take(2 * NS * Npc);
          L.o_maps = take(8 * sizeof(CUtensorMap));
          L.o_ex = take(4 * (Npc / 64));
        } else {
          L.o_s1 = take(8 * Npc);
          L.o_s2 = take(8 * Npc);
          L.o_s3 = take(8 * Npc);
          L.o_cr = take(8 * (size_t)L.px->n * L.py->n);
        }
        if (d.mir) {
          L.o_lx = take(4 * (size_t)L.px->np);
          L.o_ly = take(4 * (size_t)L.py->np);
          L.o_g = take(2 * 4 * (size_t)L.px->n * L.py->n);
        }
        if (low) {
          L.o_lh = take(4 * 2 * (size_t)kLowM * kLowM * (L.py->np / 128));  // G shares
          L.o_ljt = take(2 * (size_t)kLowNS * L.px->np * kLowK3);
          L.o_ljte = take((size_t)L.px->np);
          L.o_lz = take(2 * 4 * (size_t)L.px->n * L.py->n);
          L.o_lmaps = take(4 * sizeof(CUtensorMap));
        }
        tl.push_back(L);
      }
  }
  s.bytes = off;
  if (size_only) return EXT_OK;
  if (arena) {
    s.arena = arena;
  } else if (cudaMalloc(&s.arena, s.bytes) != cudaSuccess) {
    cudaGetLastError();
    s.arena = nullptr;
    g_last_error = "cudaMalloc of solve workspace failed";
    return EXT_ENOMEM;
  }
  char* A = s.arena;
  d.b = (double*)(A + o_b);
  d.xhi = (float*)(A + o_x);
  d.xlo = (float*)(A + o_xl);  // own 256-byte aligned slot: the update kernel loads float4
  d.part = (double*)(A + o_part);
  d.pq_part = (double*)(A + o_pqp);
  d.r = (float*)(A + o_r);
  d.p[0] = (float*)(A + o_p0);
  d.p[1] = (float*)(A + o_p1);
  d.q = (float*)(A + o_q);
  d.z = (float*)(A + o_z);
  d.r_lo = (float*)(A + o_rl);
  d.p_lo[0] = (float*)(A + o_p0l);
  d.p_lo[1] = (float*)(A + o_p1l);
  d.q_lo = (float*)(A + o_ql);
  d.z_lo = (float*)(A + o_zl);
  d.mask = (uint8_t*)(A + o_mask);
  d.t1 = (float*)(A + o_t1);
  d.t2 = (float*)(A + o_t2);
  d.t3 = (float*)(A + o_t3);
  d.t1_lo = (float*)(A + o_t1l);
  d.t2_lo = (float*)(A + o_t2l);
  d.t3_lo = (float*)(A + o_t3l);
  d.st_maps = nullptr;
  if (st_copy) {
    CUtensorMap smaps[kStMaps];
    const int rc1 = make_stencil_maps(smaps, d, d.sten_ty);
    if (rc1) return rc1;
    BX_CUDA(cudaMemcpy(A + o_smaps, smaps, sizeof(smaps), cudaMemcpyHostToDevice));
    d.st_maps = A + o_smaps;
  }
  d.qx = px->q;
  d.qxt = px->qt;
  d.qy = py->q;
  d.qyt = py->qt;
  if (host_io) {
    s.phi_stage = (float*)(A + o_io);
    s.f_stage = s.phi_stage + N;
    s.out_stage = s.f_stage + N;
  }
  // eigenvalues of L_x, L_y scaled like the stencil weights, and the weight normaliser
  double a = 1.0 / (prob.hx * prob.hx), c = 1.0 / (prob.hy * prob.hy);
  const double m = std::max(a, c);
  a /= m;
  c /= m;
  std::vector<float> lx(d.nxp, 0.f), ly(d.nyp, 0.f);
  for (int k = 0; k < nx; ++k) lx[k] = (float)(px->lam[k] * a);
  for (int k = 0; k < ny; ++k) ly[k] = (float)(py->lam[k] * c);
  double smin;
  // smallest nonzero eigenvalue sum: min over the two axes' smallest entries
  double mx0 = 1e300, mx1 = 1e300, my0 = 1e300, my1 = 1e300;  // smallest, smallest nonzero
  for (int k = 0; k < nx; ++k) {
    const double v = (float)(px->lam[k] * a);
    mx0 = std::min(mx0, v);
    if (v > 0) mx1 = std::min(mx1, v);
  }
  for (int k = 0; k < ny; ++k) {
    const double v = (float)(py->lam[k] * c);
    my0 = std::min(my0, v);
    if (v > 0) my1 = std::min(my1, v);
  }
  smin = mx0 + my0;
  if (!(smin > 0)) smin = std::min(mx0 + my1, mx1 + my0);
  d.wnorm = (float)(smin * smin);
  d.zero_mode = (prob.bc_x != EXT_BC_DIRICHLET && prob.bc_y != EXT_BC_DIRICHLET);
  d.lamx = (const float*)(A + o_lx);
  d.lamy = (const float*)(A + o_ly);
  BX_CUDA(cudaMemcpy(A + o_lx, lx.data(), 4 * lx.size(), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy(A + o_ly, ly.data(), 4 * ly.size(), cudaMemcpyHostToDevice));
  // the transform problems
  const bool bf = ctx->split == 1;
  for (const TcLay& L : tl) {
    SlotDesc t = d;  // the slot's fields; a class problem overrides its domain and operands below
    PlanDev* qx = L.px;
    PlanDev* qy = L.py;
    if (!ctx->tc) {
      // a class problem on the CUDA cores: its residual (formed by the fold kernel), T1..T3, the
      // class bases as double-float planes, its eigenvalues and its result g
      t.nx = qx->n;
      t.ny = qy->n;
      t.nxp = qx->np;
      t.nyp = qy->np;
      t.n_gm_tiles = (t.nxp / 128) * (t.nyp / 64);
      t.mir = 0;
      t.mir_out = 1;
      t.mask = nullptr;
      t.b = nullptr;
      t.xhi = t.xlo = nullptr;
      t.q = t.q_lo = nullptr;
      t.p[0] = t.p[1] = t.p_lo[0] = t.p_lo[1] = nullptr;
      t.part = t.pq_part = nullptr;
      t.st_maps = nullptr;
      const size_t Npc = (size_t)t.nxp * t.nyp, nc = (size_t)t.nx * t.ny;
      t.t1 = (float*)(A + L.o_s1);
      t.t1_lo = t.t1 + Npc;
      t.t2 = (float*)(A + L.o_s2);
      t.t2_lo = t.t2 + Npc;
      t.t3 = (float*)(A + L.o_s3);
      t.t3_lo = t.t3 + Npc;
      t.r = (float*)(A + L.o_cr);
      t.r_lo = t.r + nc;
      t.qx = qx->q;
      t.qxt = qx->qt;
      t.qy = qy->q;
      t.qyt = qy->qt;
      t.z = (float*)(A + L.o_g);
      t.z_lo = t.z + nc;
      std::vector<float> lxc(t.nxp, 0.f), lyc(t.nyp, 0.f);
      for (int k = 0; k < t.nx; ++k) lxc[k] = (float)(qx->lam[k] * a);
      for (int k = 0; k < t.ny; ++k) lyc[k] = (float)(qy->lam[k] * c);
      BX_CUDA(cudaMemcpy(A + L.o_lx, lxc.data(), 4 * lxc.size(), cudaMemcpyHostToDevice));
      BX_CUDA(cudaMemcpy(A + L.o_ly, lyc.data(), 4 * lyc.size(), cudaMemcpyHostToDevice));
      t.lamx = (const float*)(A + L.o_lx);
      t.lamy = (const float*)(A + L.o_ly);
      t.lowm_x = t.lowm_y = 0;
      s.tcp[L.c] = t;
      continue;
    }
    int rc2 = ensure_tc_plan(ctx, qx);
    if (!rc2) rc2 = ensure_tc_plan(ctx, qy);
    if (rc2) return rc2;
    if (d.mir) {
      t.nx = qx->n;
      t.ny = qy->n;
      t.nxp = qx->np;
      t.nyp = qy->np;
      t.n_gm_tiles = t.n_tc_tiles = (t.nxp / 128) * (t.nyp / 64);
      t.mir = 0;
      t.mir_out = 1;
      // only the transform fields are live: grid vectors of the slot stay out of reach
      t.mask = nullptr;
      t.b = nullptr;
      t.xhi = t.xlo = nullptr;
      t.r = t.r_lo = t.q = t.q_lo = nullptr;
      t.p[0] = t.p[1] = t.p_lo[0] = t.p_lo[1] = nullptr;
      t.part = t.pq_part = nullptr;
      t.t1 = t.t2 = t.t3 = t.t1_lo = t.t2_lo = t.t3_lo = nullptr;
      t.st_maps = nullptr;
      t.z = (float*)(A + L.o_g);  // the class result g, [ny][nx] hi then lo
      t.z_lo = t.z + (size_t)t.nx * t.ny;
      std::vector<float> lxc(t.nxp, 0.f), lyc(t.nyp, 0.f);
      for (int k = 0; k < t.nx; ++k) lxc[k] = (float)(qx->lam[k] * a);
      for (int k = 0; k < t.ny; ++k) lyc[k] = (float)(qy->lam[k] * c);
      BX_CUDA(cudaMemcpy(A + L.o_lx, lxc.data(), 4 * lxc.size(), cudaMemcpyHostToDevice));
      BX_CUDA(cudaMemcpy(A + L.o_ly, lyc.data(), 4 * lyc.size(), cudaMemcpyHostToDevice));
      t.lamx = (const float*)(A + L.o_lx);
      t.lamy = (const float*)(A + L.o_ly);
    }
    const size_t Npc = (size_t)t.nxp * t.nyp, nex = Npc / 64;
    t.tc_r = A + L.o_tr;
    t.tc_t1 = A + L.o_tt1;
    t.tc_t2 = A + L.o_tt2;
    t.tc_t3 = A + L.o_tt3;
    t.tmaps = A + L.o_maps;
    for (int k = 0; k < 4; ++k) t.tc_e[k] = (int8_t*)(A + L.o_ex + k * nex);
    t.tc_eb[0] = plan_exps(qx, 1);  // Qx^T rows
    t.tc_eb[1] = plan_exps(qy, 1);  // Qy^T rows
    t.tc_eb[2] = plan_exps(qx, 0);  // Qx rows
    t.tc_eb[3] = plan_exps(qy, 0);  // Qy rows
    BX_CUDA(cudaMemset(t.tc_r, 0, 2 * (low ? kLowNS : NS) * Npc));
    BX_CUDA(cudaMemset(A + L.o_ex, 0, 4 * nex));
    CUtensorMap maps[8];
    const size_t pxp = (size_t)t.nxp * t.nxp, pyp = (size_t)t.nyp * t.nyp;
    uint16_t* qxb = (uint16_t*)qx->tc;
    uint16_t* qyb = (uint16_t*)qy->tc;
    // A operands: r planes [P][nyp][nxp], T1 [P][nxp][nyp], T2 [P][nyp][nxp], T3 [P][nxp][nyp]
    int rc3 = make_tmap(&maps[0], t.tc_r, bf, t.nxp, (uint64_t)NS * t.nyp, 128);
    if (!rc3) rc3 = make_tmap(&maps[1], t.tc_t1, bf, t.nyp, (uint64_t)NS * t.nxp, 128);
    if (!rc3) rc3 = make_tmap(&maps[2], t.tc_t2, bf, t.nxp, (uint64_t)NS * t.nyp, 128);
    if (!rc3) rc3 = make_tmap(&maps[3], t.tc_t3, bf, t.nyp, (uint64_t)NS * t.nxp, 128);
    // B operands: Qx^T, Qy^T, Qx, Qy planes
    if (!rc3) rc3 = make_tmap(&maps[4], qxb + NS * pxp, bf, t.nxp, (uint64_t)NS * t.nxp, 64);
    if (!rc3) rc3 = make_tmap(&maps[5], qyb + NS * pyp, bf, t.nyp, (uint64_t)NS * t.nyp, 64);
    if (!rc3) rc3 = make_tmap(&maps[6], qxb, bf, t.nxp, (uint64_t)NS * t.nxp, 64);
    if (!rc3) rc3 = make_tmap(&maps[7], qyb, bf, t.nyp, (uint64_t)NS * t.nyp, 64);
    if (rc3) return rc3;
    BX_CUDA(cudaMemcpy(A + L.o_maps, maps, sizeof(maps), cudaMemcpyHostToDevice));
    t.lowm_x = t.lowm_y = 0;
    if (low) {
      t.lowm_x = std::min(kLowM, t.nx);
      t.lowm_y = std::min(kLowM, t.ny);
      t.low_gp = (float*)(A + L.o_lh);
      t.low_jt = A + L.o_ljt;
      t.low_jt_e = (int8_t*)(A + L.o_ljte);
      t.low_z = (float*)(A + L.o_lz);
      const char* lxp = (const char*)qx->low;
      const char* lyp = (const char*)qy->low;
      t.low_qxd = (const float*)(lxp + qx->low_off_d);
      t.low_qyd = (const float*)(lyp + qy->low_off_d);
      t.low_qxt_e = (const int8_t*)(lxp + qx->low_off_te);
      t.low_qy_e = (const int8_t*)(lyp + qy->low_off_qe);
      t.n_l1_tiles = t.nyp / 128;
      t.n_l3_tiles = t.nxp / 128;  // inverse product: one item per 128 rows of x
      CUtensorMap lm[4];
      int rc4 = make_tmap(&lm[0], t.tc_r, bf, t.nxp, (uint64_t)kLowNS * t.nyp, 128);
      if (!rc4) rc4 = make_tmap(&lm[1], qx->low, bf, t.nxp, (uint64_t)kLowNS * kLowM, kLowM);
      if (!rc4) rc4 = make_tmap(&lm[2], t.low_jt, bf, kLowK3, (uint64_t)kLowNS * t.nxp, 128);
      if (!rc4) rc4 = make_tmap(&lm[3], (char*)qy->low + qy->low_off_q, bf, kLowK3, (uint64_t)kLowNS * t.nyp, kLowM);
      if (rc4) return rc4;
      BX_CUDA(cudaMemcpy(A + L.o_lmaps, lm, sizeof(lm), cudaMemcpyHostToDevice));
      t.low_maps = A + L.o_lmaps;
    }
    s.tcp[L.c] = t;
  }
  s.n_tcp = (int)tl.size();
  if (ctx->tc && !d.mir) d = s.tcp[0];  // the slot is its own problem (k_tc_prepare reads it)
  if (!ctx->tc && !d.mir) {             // the slot's own transforms on the CUDA cores
    s.tcp[0] = d;
    s.n_tcp = 1;
  }
  return EXT_OK;
}

// The slot's scalars, in the slot descriptor and in each of its tensor-core problems.
static void set_slot_scalars(SlotHost& s, SlotScalars* sc) {
  s.d.sc = sc;
  for (int c = 0; c < kMirClasses; ++c) s.tcp[c].sc = sc;
}

// Work items of the tensor-core problems of slot i (problem index kMirClasses * i + c).
static void tc_items(const SlotHost& s, int i, std::vector<WorkItem>& gm, std::vector<WorkItem>& l1,
                     std::vector<WorkItem>& l3, std::vector<WorkItem>& tcl) {
  for (int c = 0; c < kMirClasses; ++c) {
    if (s.d.mir == 0 && c > 0) break;
    if (((c & 1) && !(s.d.mir & 1)) || ((c & 2) && !(s.d.mir & 2))) continue;
    const SlotDesc& t = s.tcp[c];
    const int k = kMirClasses * i + c;
    for (int tt = 0; tt < t.n_gm_tiles; ++tt) gm.push_back({k, tt});
    if (t.lowm_x) {
      for (int tt = 0; tt < t.n_l1_tiles; ++tt) l1.push_back({k, tt});
      for (int tt = 0; tt < t.n_l3_tiles; ++tt) l3.push_back({k, tt});
    }
    tcl.push_back({k, 0});
  }
}

// Tensor-core work items in the order the persistent kernels take them: decreasing k extent of
// their transform problem (a tile's cost is proportional to it), so that the persistent CTAs of a
// launch end together; tiles of one problem keep their order.  Any order gives the same results:
// tile partial sums are stored per tile and reduced in tile order.
static void longest_first_tc(std::vector<WorkItem>& gm, const std::vector<SlotHost>& slots) {
  std::stable_sort(gm.begin(), gm.end(), [&](const WorkItem& a, const WorkItem& b) {
    const SlotDesc& da = slots[a.slot / kMirClasses].tcp[a.slot % kMirClasses];
    const SlotDesc& db = slots[b.slot / kMirClasses].tcp[b.slot % kMirClasses];
    return std::max(da.nxp, da.nyp) > std::max(db.nxp, db.nyp);
  });
}

template <class T>
static int upload(T** dst, const std::vector<T>& v) {
  BX_CUDA(cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, v.size())));
  if (!v.empty()) BX_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return EXT_OK;
}

static int build_workspace(ext_ctx* ctx, int count, const ext_problem* probs, bool host_io,
                           Workspace** out) {
  std::unique_ptr<Workspace> W(new Workspace());
  W->key = shape_key(count, probs, host_io);
  W->host_io = host_io;
  W->slots.resize(count);
  std::vector<WorkItem> st, vec, gm, l1, l3, fold, unfold, tcl, prep;
  long long call_nodes = 0;
  for (int i = 0; i < count; ++i) call_nodes += (long long)probs[i].nx * probs[i].ny;
  for (int i = 0; i < count; ++i) {
    SlotHost& s = W->slots[i];
    int rc = build_slot(ctx, probs[i], host_io, s, nullptr, false, call_nodes >= kLowAutoNodes);
    if (rc) {
      for (int j = 0; j < i; ++j) cudaFree(W->slots[j].arena);
      cudaFree(s.arena);
      return rc;
    }
    SlotDesc& d = s.d;
    if (d.aniso) W->aniso = true;
    for (int t = 0; t < d.n_st_tiles; ++t) st.push_back({i, t});
    for (int t = 0; t < d.n_vec_items; ++t) vec.push_back({i, t});
    tc_items(s, i, gm, l1, l3, tcl);
    for (int t = 0; t < d.n_fold_items; ++t) fold.push_back({i, t});
    for (int t = 0; t < d.n_unfold_tiles; ++t) unfold.push_back({i, t});
    if (ctx->tc && !d.mir)
      for (int t = 0; t < d.n_prep_items; ++t) prep.push_back({i, t});
  }
  longest_first_tc(gm, W->slots);
  std::vector<WorkItem> sl;
  for (int i = 0; i < count; ++i) sl.push_back({i, 0});
  W->n_sl = (int)sl.size();
  W->n_st = (int)st.size();
  W->n_vec = (int)vec.size();
  W->n_gm = (int)gm.size();
  BX_CUDA(cudaMalloc(&W->d_sc, sizeof(SlotScalars) * count));
  BX_CUDA(cudaMemset(W->d_sc, 0, sizeof(SlotScalars) * count));
  BX_CUDA(cudaMallocHost(&W->h_sc, sizeof(SlotScalars) * count));
  for (int i = 0; i < count; ++i) set_slot_scalars(W->slots[i], W->d_sc + i);
  std::vector<SlotDesc> descs(count), tcps(kMirClasses * count);
  for (int i = 0; i < count; ++i) {
    descs[i] = W->slots[i].d;
    for (int c = 0; c < kMirClasses; ++c) tcps[kMirClasses * i + c] = W->slots[i].tcp[c];
  }
  int rc = upload(&W->d_slots, descs);
  if (!rc) rc = upload(&W->d_tcp, tcps);
  if (!rc) rc = upload(&W->d_st, st);
  if (!rc) rc = upload(&W->d_vec, vec);
  if (!rc) rc = upload(&W->d_gm, gm);
  if (!rc) rc = upload(&W->d_sl, sl);
  if (!rc) rc = upload(&W->d_sten, st);
  if (!rc) rc = upload(&W->d_l1, l1);
  if (!rc) rc = upload(&W->d_l3, l3);
  if (!rc) rc = upload(&W->d_fold, fold);
  if (!rc) rc = upload(&W->d_unfold, unfold);
  if (!rc) rc = upload(&W->d_tcl, tcl);
  if (!rc) rc = upload(&W->d_prep, prep);
  if (rc) return rc;
  W->n_sten = W->n_st;
  W->n_l1 = (int)l1.size();
  W->n_l3 = (int)l3.size();
  W->n_fold = (int)fold.size();
  W->n_unfold = (int)unfold.size();
  W->n_tcl = (int)tcl.size();
  W->n_prep = (int)prep.size();
  int counts[11] = {W->n_st, W->n_vec, W->n_gm, W->n_sl, W->n_sten, W->n_l1, W->n_l3,
                    W->n_fold, W->n_unfold, W->n_tcl, W->n_prep};
  BX_CUDA(cudaMalloc(&W->d_counts, sizeof(counts)));
  BX_CUDA(cudaMemcpy(W->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMalloc(&W->d_phis, sizeof(void*) * count));
  BX_CUDA(cudaMalloc(&W->d_fs, sizeof(void*) * count));
  BX_CUDA(cudaMalloc(&W->d_outs, sizeof(void*) * count));
  BX_CUDA(cudaMalloc(&W->d_dirs, sizeof(int) * count));
  BX_CUDA(cudaMallocHost(&W->h_ptrs, (3 * sizeof(void*) + sizeof(int)) * count));
  *out = W.release();
  return EXT_OK;
}

static int get_workspace(ext_ctx* ctx, int count, const ext_problem* probs, bool host_io,
                         Workspace** out) {
  const std::string key = shape_key(count, probs, host_io);
  auto it = ctx->ws.find(key);
  if (it != ctx->ws.end()) {
    *out = it->second;
    return EXT_OK;
  }
  // keep the cache small: drop everything else when it grows
  if (ctx->ws.size() >= 8) {
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->ws) free_workspace(kv.second);
    ctx->ws.clear();
  }
  Workspace* W = nullptr;
  int rc = build_workspace(ctx, count, probs, host_io, &W);
  if (rc) return rc;
  ctx->ws[key] = W;
  *out = W;
  return EXT_OK;
}

static LaunchCfg cfg_of(ext_ctx* ctx, Workspace* W, int which) {
  LaunchCfg c;
  c.wait_cycles = ctx->opt.wait_cycles;
  c.slots = W->d_slots;
  c.tcp = W->d_tcp;
  c.stream = W->stream ? W->stream : ctx->stream;
  const int cap = ctx->sm_count * 8;
  if (which == 7 || which == 8) {
    c.items = which == 7 ? W->d_fold : W->d_unfold;
    c.n_items = W->d_counts + which;
    c.grid = std::max(1, std::min(which == 7 ? W->n_fold : W->n_unfold, cap));
  } else if (which == 9) {
    c.items = W->d_tcl;
    c.n_items = W->d_counts + 9;
    c.grid = std::max(1, std::min(W->n_tcl, cap));
  } else if (which == 10) {
    c.items = W->d_prep;
    c.n_items = W->d_counts + 10;
    c.grid = std::max(1, std::min(W->n_prep, cap));
  } else if (which == 0) {
    c.items = W->d_st;
    c.n_items = W->d_counts + 0;
    c.grid = std::max(1, std::min(W->n_st, cap));
  } else if (which == 1) {
    c.items = W->d_vec;
    c.n_items = W->d_counts + 1;
    c.grid = std::max(1, std::min(W->n_vec, cap));
  } else if (which == 3) {
    c.items = W->d_sl;
    c.n_items = W->d_counts + 3;
    c.grid = std::max(1, std::min(W->n_sl, cap));
  } else if (which == 5 || which == 6) {
    c.items = which == 5 ? W->d_l1 : W->d_l3;
    c.n_items = W->d_counts + which;
    c.grid = std::max(1, std::min(which == 5 ? W->n_l1 : W->n_l3, ctx->sm_count));
  } else if (which == 4) {
    // persistent: the resident blocks, each double-buffering its tiles
    c.items = W->d_sten;
    c.n_items = W->d_counts + 4;
    c.grid = std::max(1, std::min(W->n_sten, ctx->sm_count * stencil_blocks_per_sm(W->sten_ty)));
  } else {
    c.items = W->d_gm;
    c.n_items = W->d_counts + 2;
    c.grid = std::max(1, std::min(W->n_gm, ctx->sm_count * 2));
  }
  return c;
}

static cudaEvent_t ev_get(ext_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch one kernel (fn), counting it; in profiling mode bracket it with CUDA events on the
// context's stream.  Never used while a graph is being captured with profiling on.
template <class F>
static void timed(ext_ctx* ctx, int kind, F&& fn, cudaStream_t st = nullptr) {
  ctx->launches += 1;
  if (!ctx->opt.profile) {
    fn();
    return;
  }
  if (!st) st = ctx->stream;
  cudaEvent_t a = ev_get(ctx), b = ev_get(ctx);
  // under stream capture the records must be external to become timing nodes of the graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  cudaEventRecordWithFlags(a, st, flags);
  fn();
  cudaEventRecordWithFlags(b, st, flags);
  ctx->pending.push_back({kind, a, b});
}

// Elapsed time of event pairs that are nodes of a replayed graph (the events stay owned by it).
static void harvest_graph(ext_ctx* ctx, const std::vector<Workspace::Ev>& ev) {
  for (const auto& p : ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->prof_ms[p.kind] += ms;
      ctx->prof_n[p.kind] += 1;
    }
  }
  cudaGetLastError();
}

// After a stream synchronisation: fold the recorded event pairs into the per-kind totals.
static void harvest(ext_ctx* ctx) {
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->prof_ms[p.kind] += ms;
      ctx->prof_n[p.kind] += 1;
    }
    ctx->ev_pool.push_back(p.a);
    ctx->ev_pool.push_back(p.b);
  }
  ctx->pending.clear();
  cudaGetLastError();
}

static void launch_prec(ext_ctx* ctx, Workspace* W, int mode) {
  LaunchCfg g = cfg_of(ctx, W, 2);
  if (ctx->tc) {
    // residual slices: unfolded slots directly, folded slots per mirror class
    if (W->n_prep > 0)
      timed(ctx, EXT_KERNEL_SPLIT, [&] { launch_prec_tc_prepare(cfg_of(ctx, W, 10), mode, ctx->split); },
            g.stream);
    if (W->n_fold > 0)
      timed(ctx, EXT_KERNEL_FOLD, [&] { launch_tc_fold(cfg_of(ctx, W, 7), mode, ctx->split); }, g.stream);
    // the transform kernels run over the tensor-core problems
    g.slots = W->d_tcp;
    g.grid = std::max(1, std::min(W->n_gm, ctx->sm_count));
    if (W->n_l1 > 0) {
      // the lowest modes in high precision: forward product, middle, inverse product
      LaunchCfg c1 = cfg_of(ctx, W, 5), cm = cfg_of(ctx, W, 6), c3 = cfg_of(ctx, W, 6);
      c1.slots = cm.slots = c3.slots = W->d_tcp;
      cm.grid = std::max(1, std::min(W->n_l3, ctx->sm_count * 8));  // the middle: small blocks
      timed(ctx, EXT_KERNEL_LOW_FWD, [&] { launch_low_tc(c1, 0, mode, ctx->split, ctx->d_err); }, g.stream);
      timed(ctx, EXT_KERNEL_LOW_MID, [&] { launch_low_mid(cm, mode, ctx->split); }, g.stream);
      timed(ctx, EXT_KERNEL_LOW_INV, [&] { launch_low_tc(c3, 1, mode, ctx->split, ctx->d_err); }, g.stream);
    }
  }
  if (!ctx->tc) {
    // CUDA-core transforms over the transform problems: a folded slot's classes get their
    // residuals from the fold first
    g.slots = W->d_tcp;
    if (W->n_unfold > 0)
      timed(ctx, EXT_KERNEL_FOLD, [&] { launch_simt_fold(cfg_of(ctx, W, 8), mode); }, g.stream);
  }
  for (int s = 0; s < 4; ++s) {
    timed(ctx, EXT_KERNEL_PREC0 + s, [&] {
      if (!ctx->tc) launch_prec_simt(g, s, mode);
      else launch_prec_tc(g, s, mode, ctx->split, ctx->d_err);
    }, g.stream);
  }
  if (W->n_unfold > 0)
    timed(ctx, EXT_KERNEL_UNFOLD, [&] { launch_unfold(cfg_of(ctx, W, 8), mode); }, g.stream);
  const LaunchCfg f = cfg_of(ctx, W, 3);  // one block per slot
  timed(ctx, EXT_KERNEL_PREC_FINISH, [&] { launch_prec_finish(f, mode); }, f.stream);
}

static void enqueue_iterations(ext_ctx* ctx, Workspace* W, int iters) {
  const LaunchCfg st = cfg_of(ctx, W, 0), vc = cfg_of(ctx, W, 1);
  const LaunchCfg sc = cfg_of(ctx, W, 4);
  for (int i = 0; i < iters; ++i) {
    timed(ctx, EXT_KERNEL_STENCIL, [&] { launch_stencil(sc, W->aniso, W->sten_ty, ctx->d_err); }, st.stream);
    const LaunchCfg pf = cfg_of(ctx, W, 3);  // one block per slot
    timed(ctx, EXT_KERNEL_PQ_FINISH, [&] { launch_pq_finish(pf); }, st.stream);
    timed(ctx, EXT_KERNEL_UPDATE, [&] { launch_update(vc); }, st.stream);
    launch_prec(ctx, W, 0);
  }
  timed(ctx, EXT_KERNEL_TRUE_RESIDUAL, [&] { launch_true_residual(st); }, st.stream);
  launch_prec(ctx, W, 1);
}

static int ensure_graph(ext_ctx* ctx, Workspace* W) {
  // with profiling on, the graph holds an event-record node before and after every kernel
  const int G = ctx->opt.iters_per_launch;
  if (W->graph && W->graph_iters == G) return EXT_OK;
  if (W->graph) {
    cudaGraphExecDestroy(W->graph);
    W->graph = nullptr;
  }
  cudaGraph_t g;
  if (ctx->opt.profile) {
    // events for the graph's timing nodes are created before capture begins
    const size_t need = 2 * (size_t)(8 * G + 16);
    while (ctx->ev_pool.size() < need) {
      cudaEvent_t e = nullptr;
      BX_CUDA(cudaEventCreate(&e));
      ctx->ev_pool.push_back(e);
    }
  }
  cudaStream_t cstream = W->stream ? W->stream : ctx->stream;
  BX_CUDA(cudaStreamBeginCapture(cstream, cudaStreamCaptureModeThreadLocal));
  const int64_t before = ctx->launches.load();
  const size_t pend0 = ctx->pending.size();
  enqueue_iterations(ctx, W, G);
  W->graph_nodes = ctx->launches - before;
  ctx->launches = before;  // captured, not launched
  W->graph_events.assign(ctx->pending.begin() + pend0, ctx->pending.end());
  ctx->pending.resize(pend0);
  cudaError_t e = cudaStreamEndCapture(cstream, &g);
  if (e != cudaSuccess) {
    g_last_error = std::string("graph capture: ") + cudaGetErrorString(e);
    return EXT_ECUDA;
  }
  e = cudaGraphInstantiate(&W->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    g_last_error = std::string("graph instantiate: ") + cudaGetErrorString(e);
    return EXT_ECUDA;
  }
  W->graph_iters = G;
  return EXT_OK;
}

// ---- stencil tile shape and its autotuner ----------------------------------------------------
// Re-tile the stencil of every slot of W with tiles 64 x ty: the work list, the tile counts and
// the tensor maps' box heights.  The p.q partials do not depend on the tile (64 x 16 node
// blocks), so any shape gives the same results.
static int set_stencil_shape(ext_ctx* ctx, Workspace* W, int ty) {
  if (W->sten_ty == ty) return EXT_OK;
  cudaStream_t s = W->stream ? W->stream : ctx->stream;
  BX_CUDA(cudaStreamSynchronize(s));
  std::vector<WorkItem> sten;
  std::vector<SlotDesc> descs;
  for (int i = 0; i < (int)W->slots.size(); ++i) {
    SlotDesc& d = W->slots[i].d;
    d.sten_ty = ty;
    d.n_sten_tiles = ((d.nx + kStTileX - 1) / kStTileX) * ((d.ny + ty - 1) / ty);
    for (int t = 0; t < d.n_sten_tiles; ++t) sten.push_back({i, t});
    if (d.st_maps) {
      CUtensorMap m[kStMaps];
      const int rc = make_stencil_maps(m, d, ty);
      if (rc) return rc;
      BX_CUDA(cudaMemcpy(const_cast<void*>(d.st_maps), m, sizeof(m), cudaMemcpyHostToDevice));
    }
    descs.push_back(d);
  }
  cudaFree(W->d_sten);
  W->d_sten = nullptr;
  BX_CUDA(cudaMalloc(&W->d_sten, sizeof(WorkItem) * sten.size()));
  BX_CUDA(cudaMemcpy(W->d_sten, sten.data(), sizeof(WorkItem) * sten.size(), cudaMemcpyHostToDevice));
  W->n_sten = (int)sten.size();
  BX_CUDA(cudaMemcpy(W->d_counts + 4, &W->n_sten, sizeof(int), cudaMemcpyHostToDevice));
  BX_CUDA(cudaMemcpy(W->d_slots, descs.data(), sizeof(SlotDesc) * descs.size(), cudaMemcpyHostToDevice));
  W->sten_ty = ty;
  if (W->graph) {
    cudaGraphExecDestroy(W->graph);
    W->graph = nullptr;
  }
  return EXT_OK;
}

// Tuning results by workspace shape, shared by the contexts of the process and, when the
// environment variable EXT_TUNE_CACHE names a file, kept there (one "key tile_y" line each).
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const Workspace* W) {
  char buf[32];
  snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)std::hash<std::string>{}(W->key));
  return buf;
}

int tune_lookup(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tune_loaded) {
    g_tune_loaded = true;
    if (const char* path = std::getenv("EXT_TUNE_CACHE")) {
      if (FILE* f = std::fopen(path, "r")) {
        char k[64];
        int ty = 0;
        while (std::fscanf(f, "%63s %d", k, &ty) == 2)
          if (ty == 16 || ty == 32) g_tune[k] = ty;
        std::fclose(f);
      }
    }
  }
  auto it = g_tune.find(key);
  return it == g_tune.end() ? 0 : it->second;
}

void tune_store(const std::string& key, int ty) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = ty;
  if (const char* path = std::getenv("EXT_TUNE_CACHE")) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%s %d\n", key.c_str(), ty);
      std::fclose(f);
    }
  }
}
}  // namespace

// Choose the stencil tile height of W: from the cache, or by timing each candidate on the
// workspace's own slots right after their set-up (iteration 0: beta = 0 and z = 0, so the
// launches write zeros that the first iteration overwrites).
static int autotune_stencil(ext_ctx* ctx, Workspace* W) {
  const std::string key = tune_key(W);
  int ty = tune_lookup(key);
  if (!ty) {
    cudaStream_t s = W->stream ? W->stream : ctx->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BX_CUDA(cudaEventCreate(&e0));
    BX_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int cand : {32, 16}) {
      int rc = set_stencil_shape(ctx, W, cand);
      if (rc) return rc;
      const LaunchCfg sc = cfg_of(ctx, W, 4);
      launch_stencil(sc, W->aniso, cand, ctx->d_err);  // warm
      BX_CUDA(cudaEventRecord(e0, s));
      constexpr int kReps = 5;
      for (int r = 0; r < kReps; ++r) launch_stencil(sc, W->aniso, cand, ctx->d_err);
      BX_CUDA(cudaEventRecord(e1, s));
      BX_CUDA(cudaEventSynchronize(e1));
      ctx->launches += kReps + 1;
      float ms = 0.f;
      BX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        ty = cand;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_store(key, ty);
  }
  W->tuned = true;
  return set_stencil_shape(ctx, W, ty);
}

// Relative A-norm error estimate of the returned iterate from the CG step terms alpha_j rho_j.
static double err_estimate(const SlotScalars& sc) {
  if (!(sc.aro_total > 0.0)) return 0.0;
  double tail = 0.0;
  const int n = std::min(sc.aro_n, kErrDelay);
  for (int i = 0; i < n; ++i) tail += sc.aro_ring[i];
  return std::sqrt(tail / sc.aro_total);
}

static int map_status(int st, int n_known, const ext_problem& p) {
  if (st == ST_OK && n_known == 0 && p.bc_x != EXT_BC_DIRICHLET && p.bc_y != EXT_BC_DIRICHLET)
    return EXT_ENOKNOWN;
  return st;
}

// Full solve of the slots of W (inputs already bound); writes outputs and results.
static int run_solve(ext_ctx* ctx, Workspace* W, const float* const* phis, const float* const* fs,
                     float* const* outs, const int* dirs, ext_result* results,
                     double* out64 = nullptr) {
  const auto t0 = std::chrono::steady_clock::now();
  const int count = (int)W->slots.size();
  cudaStream_t s = ctx->stream;
  // bind inputs (staging host arrays when needed)
  char* hp = (char*)W->h_ptrs;
  const float** h_phis = (const float**)hp;
  const float** h_fs = h_phis + count;
  float** h_outs = (float**)(h_fs + count);
  int* h_dirs = (int*)(h_outs + count);
  for (int i = 0; i < count; ++i) {
    SlotHost& sl = W->slots[i];
    const size_t N = (size_t)sl.prob.nx * sl.prob.ny;
    if (W->host_io) {
      BX_CUDA(cudaMemcpyAsync(sl.phi_stage, phis[i], 4 * N, cudaMemcpyHostToDevice, s));
      BX_CUDA(cudaMemcpyAsync(sl.f_stage, fs[i], 4 * N, cudaMemcpyHostToDevice, s));
      h_phis[i] = sl.phi_stage;
      h_fs[i] = sl.f_stage;
      h_outs[i] = sl.out_stage;
    } else {
      h_phis[i] = phis[i];
      h_fs[i] = fs[i];
      h_outs[i] = outs[i];
    }
    h_dirs[i] = dirs[i];
  }
  BX_CUDA(cudaMemcpyAsync(W->d_phis, h_phis, sizeof(void*) * count, cudaMemcpyHostToDevice, s));
  BX_CUDA(cudaMemcpyAsync(W->d_fs, h_fs, sizeof(void*) * count, cudaMemcpyHostToDevice, s));
  BX_CUDA(cudaMemcpyAsync(W->d_outs, h_outs, sizeof(void*) * count, cudaMemcpyHostToDevice, s));
  BX_CUDA(cudaMemcpyAsync(W->d_dirs, h_dirs, sizeof(int) * count, cudaMemcpyHostToDevice, s));
  // scalars: parameters and zero counters
  for (int i = 0; i < count; ++i) {
    SlotScalars& sc = W->h_sc[i];
    memset(&sc, 0, sizeof(sc));
    const ext_problem& p = W->slots[i].prob;
    sc.rtol2 = ctx->opt.rtol * ctx->opt.rtol;
    sc.maxit = ctx->opt.maxit > 0 ? ctx->opt.maxit : 10 * std::max(p.nx, p.ny);
    sc.fold_every = ctx->opt.true_res_every;
    sc.delta2 = ctx->opt.replace_factor * ctx->opt.replace_factor;
    sc.flexible = ctx->opt.flexible;
    sc.status = ST_RUNNING;
  }
  BX_CUDA(cudaMemcpyAsync(W->d_sc, W->h_sc, sizeof(SlotScalars) * count, cudaMemcpyHostToDevice, s));
  int rc = EXT_OK;
  if (!ctx->opt.autotune) rc = set_stencil_shape(ctx, W, ctx->opt.tile_y == 16 ? 16 : 32);
  if (rc) return rc;
  timed(ctx, EXT_KERNEL_SETUP, [&] { launch_setup(cfg_of(ctx, W, 0), W->d_phis, W->d_fs, W->d_dirs); });
  timed(ctx, EXT_KERNEL_SETUP, [&] { launch_rhs_scale(cfg_of(ctx, W, 0)); });
  if (ctx->opt.autotune && !W->tuned) rc = autotune_stencil(ctx, W);
  if (rc) return rc;
  ctx->last_tile_y = W->sten_ty;
  rc = ensure_graph(ctx, W);
  if (rc) return rc;
  launch_prec(ctx, W, 1);
  BX_CUDA(cudaGetLastError());
  int max_blocks = 0;
  for (int i = 0; i < count; ++i) {
    const ext_problem& p = W->slots[i].prob;
    const int mi = ctx->opt.maxit > 0 ? ctx->opt.maxit : 10 * std::max(p.nx, p.ny);
    max_blocks = std::max(max_blocks, mi);
  }
  max_blocks = max_blocks / std::max(1, W->graph_iters) + 8;
  for (int blk = 0; blk < max_blocks; ++blk) {
    BX_CUDA(cudaGraphLaunch(W->graph, s));
    ctx->launches += W->graph_nodes;
    BX_CUDA(cudaMemcpyAsync(W->h_sc, W->d_sc, sizeof(SlotScalars) * count, cudaMemcpyDeviceToHost, s));
    BX_CUDA(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BX_CUDA(cudaStreamSynchronize(s));
    harvest(ctx);
    if (ctx->opt.profile) harvest_graph(ctx, W->graph_events);
    if (*ctx->h_err) {
      BX_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
      BX_CUDA(cudaStreamSynchronize(s));
      g_last_error = "a bounded device wait (tensor copy or tensor-core pipeline) ran out";
      return EXT_ETIMEOUT;
    }
    bool running = false;
    for (int i = 0; i < count; ++i)
      if (W->h_sc[i].status == ST_RUNNING) running = true;
    if (!running) break;
  }
  if (out64) {
    const SlotHost& sl = W->slots[0];
    timed(ctx, EXT_KERNEL_OUTPUT, [&] {
      launch_output64(W->d_slots, sl.prob.nx * sl.prob.ny, W->host_io ? sl.f_stage : fs[0], out64, s);
    });
  } else {
    timed(ctx, EXT_KERNEL_OUTPUT, [&] { launch_output(cfg_of(ctx, W, 1), W->d_fs, W->d_outs); });
  }
  BX_CUDA(cudaGetLastError());
  if (W->host_io && !out64) {
    for (int i = 0; i < count; ++i) {
      SlotHost& sl = W->slots[i];
      const size_t N = (size_t)sl.prob.nx * sl.prob.ny;
      BX_CUDA(cudaMemcpyAsync(outs[i], sl.out_stage, 4 * N, cudaMemcpyDeviceToHost, s));
    }
  }
  BX_CUDA(cudaStreamSynchronize(s));
  harvest(ctx);
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = EXT_OK;
  for (int i = 0; i < count; ++i) {
    const SlotScalars& sc = W->h_sc[i];
    const ext_problem& p = W->slots[i].prob;
    int st = sc.status == ST_RUNNING ? EXT_ETIMEOUT : map_status(sc.status, sc.n_known, p);
    if (results) {
      ext_result& r = results[i];
      r.status = st;
      r.iters = sc.it;
      r.relres_true = sc.bb > 0 ? std::sqrt(sc.rr_true / sc.bb) : 0.0;
      r.relres_rec = sc.bb > 0 ? std::sqrt(sc.rr / sc.bb) : 0.0;
      r.n_known = sc.n_known;
      r.n_unknown = p.nx * p.ny - sc.n_known;
      r.ms_queue = 0.0;
      r.ms_solve = ms;
      r.err_est = err_estimate(sc);
    }
    if (st != EXT_OK && worst == EXT_OK) worst = st;
  }
  return worst;
}

// ---------------------------------------------------------------------------------------------
// public API
// ---------------------------------------------------------------------------------------------
extern "C" {

void ext_options_default(ext_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->prec = EXT_PREC_FP32;
  o->rtol = 1e-8;
  o->maxit = 0;
  o->true_res_every = 200;
  o->replace_factor = 1e-2;
  o->iters_per_launch = 10;
  o->hbm_budget = 0;
  o->flexible = 0;
  o->max_slots = 256;
  o->autotune = 1;
  o->tile_y = 32;
  o->low_modes = 2;
  o->fold = 1;
}

const char* ext_strerror(int code) {
  switch (code) {
    case EXT_OK: return "ok";
    case EXT_PENDING: return "pending";
    case EXT_EINVAL: return "invalid argument (size, spacing, enum, null pointer or NaN in phi)";
    case EXT_ENOKNOWN: return "no known node and no Dirichlet edge: extension not unique";
    case EXT_ENOMEM: return "device allocation failed";
    case EXT_EADMIT: return "request footprint exceeds the serving HBM budget";
    case EXT_ENOTCONV: return "not converged within maxit";
    case EXT_EBREAKDOWN: return "CG breakdown (non-positive curvature or non-finite scalar)";
    case EXT_ETIMEOUT: return "bounded wait ran out";
    case EXT_ECUDA: return "CUDA runtime error";
    case EXT_ENOTSUP: return "not supported on this device";
    case EXT_ENOTFOUND: return "unknown ticket";
    default: return "unknown error code";
  }
}

const char* ext_last_error(void) { return g_last_error.c_str(); }

int ext_axis_slices(int32_t n, ext_bc bc, int32_t type, uint16_t* codes, int8_t* exps) {
  if (n < 4 || n > 32768 || bc < 0 || bc > 2 || (type != 0 && type != 1) || !codes || !exps)
    return EXT_EINVAL;
  std::vector<uint16_t> h;
  std::vector<int8_t> ex;
  slice_plan_host(n, bc, pad_to(n, kPad), type, h, ex);
  std::copy(h.begin(), h.end(), codes);
  std::copy(ex.begin(), ex.end(), exps);
  return EXT_OK;
}

int ext_axis_basis(int32_t n, ext_bc bc, double* Q, double* lam) {
  if (n < 4 || n > 32768 || bc < 0 || bc > 2 || !Q || !lam) return EXT_EINVAL;
  const AxisBasis B = make_axis_basis(n, bc);
  std::copy(B.Q.begin(), B.Q.end(), Q);
  std::copy(B.lam.begin(), B.lam.end(), lam);
  return EXT_OK;
}

int ext_axis_class_basis(int32_t n, ext_bc bc, int32_t cls, double* Q, double* lam) {
  if (n < 4 || n > 32768 || bc < 0 || bc > 2 || (cls != 0 && cls != 1) || !Q || !lam) return EXT_EINVAL;
  const AxisBasis B = make_class_basis(n, bc, cls);
  std::copy(B.Q.begin(), B.Q.end(), Q);
  std::copy(B.lam.begin(), B.lam.end(), lam);
  return EXT_OK;
}

int ext_create(const ext_options* opt, void* cuda_stream, ext_ctx** out) {
  if (!out) return EXT_EINVAL;
  *out = nullptr;
  ext_options o;
  ext_options_default(&o);
  if (opt) o = *opt;
  if (o.prec != EXT_PREC_FP32 && o.prec != EXT_PREC_MIXED_BF16 && o.prec != EXT_PREC_MIXED_FP16)
    return EXT_EINVAL;
  if (!(o.rtol > 0.0) || o.rtol >= 1.0) return EXT_EINVAL;
  if (o.iters_per_launch <= 0) o.iters_per_launch = 10;
  if (o.true_res_every <= 0) o.true_res_every = 200;
  if (!(o.replace_factor > 0.0) || o.replace_factor >= 1.0) o.replace_factor = 1e-2;
  // residual replacement happens at graph boundaries: make the period a multiple of G
  o.true_res_every = (o.true_res_every + o.iters_per_launch - 1) / o.iters_per_launch * o.iters_per_launch;
  if (o.max_slots <= 0) o.max_slots = 256;
  std::unique_ptr<ext_ctx> ctx(new ext_ctx());
  ctx->opt = o;
  BX_CUDA(cudaGetDevice(&ctx->device));
  cudaDeviceProp prop;
  BX_CUDA(cudaGetDeviceProperties(&prop, ctx->device));
  ctx->sm_count = prop.multiProcessorCount;
  ctx->cc_major = prop.major;
  ctx->cc_minor = prop.minor;
  if (o.prec != EXT_PREC_FP32 && !(prop.major == 10 && tc_supported())) return EXT_ENOTSUP;
  ctx->tc = o.prec != EXT_PREC_FP32;
  ctx->split = o.prec == EXT_PREC_MIXED_BF16 ? 1 : 0;
  if (ctx->tc) BX_CUDA(tc_init());
  BX_CUDA(stencil_init());
  BX_CUDA(cudaMalloc(&ctx->d_err, sizeof(int)));
  BX_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
  BX_CUDA(cudaMallocHost(&ctx->h_err, sizeof(int)));
  *ctx->h_err = 0;
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    BX_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  *out = ctx.release();
  return EXT_OK;
}

void ext_serve_shutdown(ext_ctx* ctx);

void ext_destroy(ext_ctx* ctx) {
  if (!ctx) return;
  ext_serve_shutdown(ctx);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->ws) free_workspace(kv.second);
  for (auto& kv : ctx->plans) {
    cudaFree(kv.second.q);
    cudaFree(kv.second.qt);
    cudaFree(kv.second.tc);
    cudaFree(kv.second.low);
  }
  harvest(ctx);
  cudaFree(ctx->d_err);
  cudaFreeHost(ctx->h_err);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int ext_solve_batch(ext_ctx* ctx, int count, const ext_problem* probs, const float* const* phi,
                    const float* const* f, float* const* out, ext_result* results) {
  if (!ctx || count <= 0 || !probs || !phi || !f || !out) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  bool any_host = false, any_dev = false;
  std::vector<int> dirs(count);
  for (int i = 0; i < count; ++i) {
    int rc = validate_problem(&probs[i]);
    if (rc) return rc;
    if (!phi[i] || !f[i] || !out[i]) return EXT_EINVAL;
    const bool d = is_device_ptr(phi[i]) && is_device_ptr(f[i]) && is_device_ptr(out[i]);
    (d ? any_dev : any_host) = true;
    dirs[i] = probs[i].dir;
  }
  if (any_host && any_dev) return EXT_EINVAL;  // one residency per call
  Workspace* W = nullptr;
  int rc = get_workspace(ctx, count, probs, any_host, &W);
  if (rc) return rc;
  return run_solve(ctx, W, phi, f, out, dirs.data(), results);
}

int ext_solve_multi(ext_ctx* ctx, const ext_problem* prob, const float* phi, int count,
                    const float* const* f, float* const* out, ext_result* results) {
  if (!ctx || !prob || !phi || count <= 0 || !f || !out) return EXT_EINVAL;
  // every field is one slot of the same shape reading the same phi: one workspace shape, one pair
  // of transform plans, and all fields iterate together in the same launches
  std::vector<ext_problem> probs(count, *prob);
  std::vector<const float*> phis(count, phi);
  return ext_solve_batch(ctx, count, probs.data(), phis.data(), f, out, results);
}

int ext_solve(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f, float* out,
              ext_result* res) {
  const float* phis[1] = {phi};
  const float* fs[1] = {f};
  float* outs[1] = {out};
  return ext_solve_batch(ctx, 1, prob, phis, fs, outs, res);
}

int ext_solve_f64(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f,
                  double* out64, ext_result* res) {
  if (!ctx || !prob || !phi || !f || !out64) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  int rc = validate_problem(prob);
  if (rc) return rc;
  if (!is_device_ptr(phi) || !is_device_ptr(f) || !is_device_ptr(out64)) return EXT_EINVAL;
  Workspace* W = nullptr;
  rc = get_workspace(ctx, 1, prob, false, &W);
  if (rc) return rc;
  const float* phis[1] = {phi};
  const float* fs[1] = {f};
  float* outs[1] = {nullptr};
  const int dirs[1] = {prob->dir};
  return run_solve(ctx, W, phis, fs, outs, dirs, res, out64);
}

// ---- three-dimensional extension --------------------------------------------------------------
static int validate_problem3(const ext_problem3* p) {
  if (!p) return EXT_EINVAL;
  if (p->nx < 4 || p->ny < 4 || p->nz < 4) return EXT_EINVAL;
  if (p->nz > 65535 || (int64_t)p->nx * p->ny * p->nz > (int64_t)1 << 30) return EXT_EINVAL;
  const double h[3] = {p->hx, p->hy, p->hz};
  for (double v : h)
    if (!(v > 0.0) || !std::isfinite(v)) return EXT_EINVAL;
  const int bc[3] = {p->bc_x, p->bc_y, p->bc_z};
  for (int b : bc)
    if (b < 0 || b > 2) return EXT_EINVAL;
  if (p->dir != 0 && p->dir != 1) return EXT_EINVAL;
  return EXT_OK;
}

// The arguments of the 3-D kernels: the axis plans (built or found in the context's cache).
static int tc3_build(ext_ctx* ctx, const Solve3Args& a, const Tc3Io& io, Tc3& t);

static int args3(ext_ctx* ctx, const ext_problem3* p, Solve3Args& a) {
  std::lock_guard<std::recursive_mutex> plk(ctx->plan_mu);
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.bc[0] = p->bc_x;
  a.bc[1] = p->bc_y;
  a.bc[2] = p->bc_z;
  a.dir = p->dir;
  a.h[0] = p->hx;
  a.h[1] = p->hy;
  a.h[2] = p->hz;
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int ax = 0; ax < 3; ++ax) {
    PlanDev* P = nullptr;
    const int rc = get_plan(ctx, n[ax], a.bc[ax], -1, &P);
    if (rc) return rc;
    a.q[ax] = P->q;
    a.qt[ax] = P->qt;
    a.np[ax] = P->np;
    a.lam[ax] = P->lam.data();
  }
  a.rtol = ctx->opt.rtol;
  a.maxit = ctx->opt.maxit;
  a.true_res_every = ctx->opt.true_res_every;
  a.replace_factor = ctx->opt.replace_factor;
  a.stream = ctx->stream;
  if (ctx->tc && p->nx % 128 == 0 && p->ny % 128 == 0 && p->nz % 128 == 0)
    a.tc_build = [ctx, &a](const Tc3Io& io, Tc3& t) { return tc3_build(ctx, a, io, t); };
  return EXT_OK;
}

// The 3-D transforms on the tensor cores (mixed modes, every side a multiple of 128).  Each of
// the six products contracts the contiguous axis of its operand and writes its result with that
// axis first, exactly the form of the 2-D stage kernels, so every product is one launch of
// k_prec_tc over a descriptor whose dimensions are the box's: with X, Y, Z the sides, the
// forward products are [Z Y][X] x Qx^T -> [X][Z Y], [X Z][Y] x Qy^T -> [Y][X Z] and
// [Y X][Z] x Qz^T -> [Z][Y X] (stage-1 form: the weights, with lam_x + lam_y of the rows folded
// into one array), the inverse ones the same with Q, the last in stage-3 form (mask, z, r.z).
// With every side a multiple of 128, each output's 128-blocks along its rows are exactly the
// next product's k-blocks, so the exponents carry over unchanged.
static int tc3_build(ext_ctx* ctx, const Solve3Args& a, const Tc3Io& io, Tc3& t) {
  const int X = a.nx, Y = a.ny, Z = a.nz;
  const size_t N3 = (size_t)X * Y * Z;
  const int NS = tc_planes(ctx->split);
  const bool bf = ctx->split == 1;
  PlanDev* P[3];
  {
    std::lock_guard<std::recursive_mutex> plk(ctx->plan_mu);
    const int n[3] = {X, Y, Z};
    for (int ax = 0; ax < 3; ++ax) {
      int rc = get_plan(ctx, n[ax], a.bc[ax], -1, &P[ax]);
      if (!rc) rc = ensure_tc_plan(ctx, P[ax]);
      if (rc) return rc;
    }
  }
  auto take = [&](size_t bytes) -> void* {
    void* v = nullptr;
    if (cudaMalloc(&v, bytes ? bytes : 1) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    t.owned.push_back(v);
    return v;
  };
  void* S0 = take(2 * (size_t)NS * N3);
  void* SA = take(2 * (size_t)NS * N3);
  void* SB = take(2 * (size_t)NS * N3);
  int8_t* E0 = (int8_t*)take(N3 / 128);
  int8_t* EA = (int8_t*)take(N3 / 128);
  int8_t* EB = (int8_t*)take(N3 / 128);
  const int tiles3 = ((Y * X) / 128) * (Z / 64);
  double* part = (double*)take(sizeof(double) * 4 * (size_t)tiles3);
  float* lam = (float*)take(sizeof(float) * ((size_t)Y * X + Z));
  SlotScalars* sc = (SlotScalars*)take(sizeof(SlotScalars));
  void* maps = take(6 * 8 * sizeof(CUtensorMap));
  SlotDesc* descs = (SlotDesc*)take(7 * sizeof(SlotDesc));
  if (!S0 || !SA || !SB || !E0 || !EA || !EB || !part || !lam || !sc || !maps || !descs) {
    g_last_error = "cudaMalloc of the 3-D tensor-core workspace failed";
    return EXT_ENOMEM;
  }
  BX_CUDA(cudaMemset(S0, 0, 2 * (size_t)NS * N3));
  BX_CUDA(cudaMemset(E0, 0, N3 / 128));
  SlotScalars hsc{};
  hsc.active = 1;
  hsc.need_prec = 1;
  BX_CUDA(cudaMemcpy(sc, &hsc, sizeof(hsc), cudaMemcpyHostToDevice));
  // eigenvalues scaled like the stencil (largest 1/h^2 = 1): lam_y + lam_x per row of the
  // weighted product ([ky][kx] flattened), lam_z per column; wnorm = (smallest nonzero sum)^2
  const double c[3] = {1.0 / (a.h[0] * a.h[0]), 1.0 / (a.h[1] * a.h[1]), 1.0 / (a.h[2] * a.h[2])};
  const double cm = std::max(c[0], std::max(c[1], c[2]));
  std::vector<float> lh((size_t)Y * X + Z);
  double lo0[3], lo1[3];
  const int nn[3] = {X, Y, Z};
  std::vector<float> la[3];
  for (int ax = 0; ax < 3; ++ax) {
    lo0[ax] = lo1[ax] = 1e300;
    la[ax].resize(nn[ax]);
    for (int k = 0; k < nn[ax]; ++k) {
      la[ax][k] = (float)(P[ax]->lam[k] * c[ax] / cm);
      lo0[ax] = std::min(lo0[ax], (double)la[ax][k]);
      if (la[ax][k] > 0) lo1[ax] = std::min(lo1[ax], (double)la[ax][k]);
    }
  }
  for (int ky = 0; ky < Y; ++ky)
    for (int kx = 0; kx < X; ++kx) lh[(size_t)ky * X + kx] = la[1][ky] + la[0][kx];
  for (int kz = 0; kz < Z; ++kz) lh[(size_t)Y * X + kz] = la[2][kz];
  BX_CUDA(cudaMemcpy(lam, lh.data(), sizeof(float) * lh.size(), cudaMemcpyHostToDevice));
  double smin = lo0[0] + lo0[1] + lo0[2];
  if (!(smin > 0))
    smin = std::min(lo1[0] + lo0[1] + lo0[2], std::min(lo0[0] + lo1[1] + lo0[2], lo0[0] + lo0[1] + lo1[2]));
  // descriptors
  SlotDesc d[7];
  for (int k = 0; k < 7; ++k) {
    d[k] = SlotDesc{};
    d[k].sc = sc;
  }
  const uint16_t* q[3] = {(const uint16_t*)P[0]->tc, (const uint16_t*)P[1]->tc, (const uint16_t*)P[2]->tc};
  const size_t pl[3] = {(size_t)X * X, (size_t)Y * Y, (size_t)Z * Z};
  auto QT = [&](int ax) { return (void*)(q[ax] + NS * pl[ax]); };  // Q^T planes follow the Q planes
  auto QQ = [&](int ax) { return (void*)q[ax]; };
  CUtensorMap m[6][8];
  memset(m, 0, sizeof(m));
  // [0]: residual slicing, rows (z, y), columns x
  d[0].nx = X; d[0].ny = Z * Y; d[0].nxp = X; d[0].nyp = Z * Y;
  d[0].r = const_cast<float*>(io.rh); d[0].r_lo = const_cast<float*>(io.rl);
  d[0].tc_r = S0; d[0].tc_e[0] = E0;
  // [1] F1 (stage-0 form): A = r slices [Z Y][X], B = Qx^T -> SA [X][Z Y]
  d[1].nyp = Z * Y; d[1].nxp = X; d[1].nx = X; d[1].ny = Z * Y;
  int rc = make_tmap(&m[0][0], S0, bf, X, (uint64_t)NS * Z * Y, 128);
  if (!rc) rc = make_tmap(&m[0][4], QT(0), bf, X, (uint64_t)NS * X, 64);
  d[1].tc_e[0] = E0; d[1].tc_eb[0] = plan_exps(P[0], 1); d[1].tc_t1 = SA; d[1].tc_e[1] = EA;
  // [2] F2 (stage-0 form): A = SA as [X Z][Y], B = Qy^T -> SB [Y][X Z]
  d[2].nyp = X * Z; d[2].nxp = Y; d[2].nx = Y; d[2].ny = X * Z;
  if (!rc) rc = make_tmap(&m[1][0], SA, bf, Y, (uint64_t)NS * X * Z, 128);
  if (!rc) rc = make_tmap(&m[1][4], QT(1), bf, Y, (uint64_t)NS * Y, 64);
  d[2].tc_e[0] = EA; d[2].tc_eb[0] = plan_exps(P[1], 1); d[2].tc_t1 = SB; d[2].tc_e[1] = EB;
  // [3] F3 (stage-1 form, weights): A = SB as [Y X][Z], B = Qz^T -> SA [Z][Y X]
  d[3].nxp = Y * X; d[3].nyp = Z; d[3].nx = Y * X; d[3].ny = Z;
  if (!rc) rc = make_tmap(&m[2][1], SB, bf, Z, (uint64_t)NS * Y * X, 128);
  if (!rc) rc = make_tmap(&m[2][5], QT(2), bf, Z, (uint64_t)NS * Z, 64);
  d[3].tc_e[1] = EB; d[3].tc_eb[1] = plan_exps(P[2], 1); d[3].tc_t2 = SA; d[3].tc_e[2] = EA;
  d[3].lamx = lam; d[3].lamy = lam + (size_t)Y * X; d[3].wnorm = (float)(smin * smin);
  // [4] I1 (stage-2 form): A = SA as [Z Y][X], B = Qx -> SB [X][Z Y]
  d[4].nyp = Z * Y; d[4].nxp = X; d[4].nx = X; d[4].ny = Z * Y;
  if (!rc) rc = make_tmap(&m[3][2], SA, bf, X, (uint64_t)NS * Z * Y, 128);
  if (!rc) rc = make_tmap(&m[3][6], QQ(0), bf, X, (uint64_t)NS * X, 64);
  d[4].tc_e[2] = EA; d[4].tc_eb[2] = plan_exps(P[0], 0); d[4].tc_t3 = SB; d[4].tc_e[3] = EB;
  // [5] I2 (stage-2 form): A = SB as [X Z][Y], B = Qy -> SA [Y][X Z]
  d[5].nyp = X * Z; d[5].nxp = Y; d[5].nx = Y; d[5].ny = X * Z;
  if (!rc) rc = make_tmap(&m[4][2], SB, bf, Y, (uint64_t)NS * X * Z, 128);
  if (!rc) rc = make_tmap(&m[4][6], QQ(1), bf, Y, (uint64_t)NS * Y, 64);
  d[5].tc_e[2] = EB; d[5].tc_eb[2] = plan_exps(P[1], 0); d[5].tc_t3 = SA; d[5].tc_e[3] = EA;
  // [6] I3 (stage-3 form): A = SA as [Y X][Z], B = Qz -> z[Z][Y X] masked, r.z per tile
  d[6].nxp = Y * X; d[6].nyp = Z; d[6].nx = Y * X; d[6].ny = Z;
  if (!rc) rc = make_tmap(&m[5][3], SA, bf, Z, (uint64_t)NS * Y * X, 128);
  if (!rc) rc = make_tmap(&m[5][7], QQ(2), bf, Z, (uint64_t)NS * Z, 64);
  if (rc) return rc;
  d[6].tc_e[3] = EA; d[6].tc_eb[3] = plan_exps(P[2], 0);
  d[6].r = const_cast<float*>(io.rh); d[6].r_lo = const_cast<float*>(io.rl);
  d[6].q = const_cast<float*>(io.qh); d[6].q_lo = const_cast<float*>(io.ql);
  d[6].z = io.zh; d[6].z_lo = io.zl; d[6].mask = const_cast<uint8_t*>(io.mask); d[6].part = part;
  BX_CUDA(cudaMemcpy(maps, m, sizeof(m), cudaMemcpyHostToDevice));
  for (int k = 1; k < 7; ++k) d[k].tmaps = (const char*)maps + (size_t)(k - 1) * 8 * sizeof(CUtensorMap);
  BX_CUDA(cudaMemcpy(descs, d, sizeof(d), cudaMemcpyHostToDevice));
  // work items: [0] 32 rows x 128 columns; the products tiles of 128 x 64 (M x N)
  static const int kForm[7] = {-1, 0, 0, 1, 2, 2, 3};
  std::vector<WorkItem> items[7];
  for (int tt = 0; tt < ((Z * Y) / 32) * (X / 128); ++tt) items[0].push_back({0, tt});
  for (int k = 1; k < 7; ++k) {
    const bool mrows_y = kForm[k] == 0 || kForm[k] == 2;  // M = nyp in the stage-0/2 forms
    const int M = mrows_y ? d[k].nyp : d[k].nxp, N = mrows_y ? d[k].nxp : d[k].nyp;
    for (int tt = 0; tt < (M / 128) * (N / 64); ++tt) items[k].push_back({k, tt});
  }
  int counts[7];
  for (int k = 0; k < 7; ++k) {
    WorkItem* di = (WorkItem*)take(sizeof(WorkItem) * items[k].size());
    if (!di) {
      g_last_error = "cudaMalloc of the 3-D tensor-core work lists failed";
      return EXT_ENOMEM;
    }
    BX_CUDA(cudaMemcpy(di, items[k].data(), sizeof(WorkItem) * items[k].size(), cudaMemcpyHostToDevice));
    t.d_items[k] = di;
    t.n_items[k] = counts[k] = (int)items[k].size();
  }
  int* dc = (int*)take(sizeof(counts));
  if (!dc) return EXT_ENOMEM;
  BX_CUDA(cudaMemcpy(dc, counts, sizeof(counts), cudaMemcpyHostToDevice));
  t.d_counts = dc;
  t.d_descs = descs;
  t.split = ctx->split;
  t.d_err = ctx->d_err;
  t.wait_cycles = ctx->opt.wait_cycles;
  t.sm_count = ctx->sm_count;
  t.part = part;
  t.n_tiles3 = counts[6];
  t.on = true;
  return EXT_OK;
}

int ext_solve3d(ext_ctx* ctx, const ext_problem3* prob, const float* phi, const float* f, float* out,
                ext_result* res) {
  if (!ctx || !prob || !phi || !f || !out) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  int rc = validate_problem3(prob);
  if (rc) return rc;
  if (!is_device_ptr(phi) || !is_device_ptr(f) || !is_device_ptr(out)) {
    g_last_error = "phi, f and out must be device pointers";
    return EXT_EINVAL;
  }
  Solve3Args a;
  rc = args3(ctx, prob, a);
  if (rc) return rc;
  ext_result r{};
  r.status = EXT_ECUDA;
  const auto t0 = std::chrono::steady_clock::now();
  std::string err;
  long long nl = 0;
  a.launches = &nl;
  rc = solve3d_run(a, phi, f, out, &r, &err);
  ctx->launches += nl;
  r.ms_solve = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (rc != EXT_OK && rc != EXT_ENOTCONV && rc != EXT_EBREAKDOWN) r.status = rc;
  if (!err.empty()) g_last_error = err;
  if (res) *res = r;
  return rc;
}

int ext_apply_biharmonic3d(ext_ctx* ctx, const ext_problem3* prob, const float* phi, const float* p,
                           float* q) {
  if (!ctx || !prob || !phi || !p || !q) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  int rc = validate_problem3(prob);
  if (rc) return rc;
  if (!is_device_ptr(phi) || !is_device_ptr(p) || !is_device_ptr(q)) return EXT_EINVAL;
  Solve3Args a;
  rc = args3(ctx, prob, a);
  if (rc) return rc;
  std::string err;
  long long nl = 0;
  a.launches = &nl;
  rc = apply3d_operator(a, phi, p, q, &err);
  ctx->launches += nl;
  if (!err.empty()) g_last_error = err;
  return rc;
}

int ext_apply_preconditioner3d(ext_ctx* ctx, const ext_problem3* prob, const float* phi, const float* r,
                               float* z, double* scale) {
  if (!ctx || !prob || !phi || !r || !z) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  int rc = validate_problem3(prob);
  if (rc) return rc;
  if (!is_device_ptr(phi) || !is_device_ptr(r) || !is_device_ptr(z)) return EXT_EINVAL;
  Solve3Args a;
  rc = args3(ctx, prob, a);
  if (rc) return rc;
  std::string err;
  long long nl = 0;
  a.launches = &nl;
  rc = apply3d_preconditioner(a, phi, r, z, scale, &err);
  ctx->launches += nl;
  if (!err.empty()) g_last_error = err;
  return rc;
}

int ext_profile_read(ext_ctx* ctx, int kinds, double* total_ms, int64_t* launches, int reset) {
  if (!ctx || kinds < 0) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  for (int k = 0; k < kinds && k < EXT_KERNEL_KINDS; ++k) {
    if (total_ms) total_ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_n[k];
  }
  if (reset) {
    for (int k = 0; k < EXT_KERNEL_KINDS; ++k) {
      ctx->prof_ms[k] = 0.0;
      ctx->prof_n[k] = 0;
    }
  }
  return EXT_OK;
}

int64_t ext_launch_count(ext_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

int ext_stencil_tile(ext_ctx* ctx, int32_t* tile_x, int32_t* tile_y) {
  if (!ctx) return EXT_EINVAL;
  if (tile_x) *tile_x = kStTileX;
  if (tile_y) *tile_y = ctx->last_tile_y;
  return EXT_OK;
}

// ---- verification entry points (device pointers) ----

static int single_setup(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f,
                        Workspace** Wout) {
  int rc = validate_problem(prob);
  if (rc) return rc;
  if (!is_device_ptr(phi) || !is_device_ptr(f)) return EXT_EINVAL;
  Workspace* W = nullptr;
  rc = get_workspace(ctx, 1, prob, false, &W);
  if (rc) return rc;
  if (!ctx->opt.autotune) rc = set_stencil_shape(ctx, W, ctx->opt.tile_y == 16 ? 16 : 32);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  const float** h_phis = (const float**)W->h_ptrs;
  const float** h_fs = h_phis + 1;
  int* h_dirs = (int*)(h_fs + 2);
  h_phis[0] = phi;
  h_fs[0] = f;
  h_dirs[0] = prob->dir;
  BX_CUDA(cudaMemcpyAsync(W->d_phis, h_phis, sizeof(void*), cudaMemcpyHostToDevice, s));
  BX_CUDA(cudaMemcpyAsync(W->d_fs, h_fs, sizeof(void*), cudaMemcpyHostToDevice, s));
  BX_CUDA(cudaMemcpyAsync(W->d_dirs, h_dirs, sizeof(int), cudaMemcpyHostToDevice, s));
  memset(W->h_sc, 0, sizeof(SlotScalars));
  W->h_sc[0].rtol2 = ctx->opt.rtol * ctx->opt.rtol;
  W->h_sc[0].maxit = 1;
  W->h_sc[0].fold_every = ctx->opt.true_res_every;
  W->h_sc[0].delta2 = 1e-4;
  BX_CUDA(cudaMemcpyAsync(W->d_sc, W->h_sc, sizeof(SlotScalars), cudaMemcpyHostToDevice, s));
  timed(ctx, EXT_KERNEL_SETUP, [&] { launch_setup(cfg_of(ctx, W, 0), W->d_phis, W->d_fs, W->d_dirs); });
  timed(ctx, EXT_KERNEL_SETUP, [&] { launch_rhs_scale(cfg_of(ctx, W, 0)); });
  BX_CUDA(cudaGetLastError());
  *Wout = W;
  return EXT_OK;
}

int ext_apply_biharmonic(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* p,
                         float* q, double* sum_pq) {
  if (!ctx || !is_device_ptr(p) || !is_device_ptr(q)) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  Workspace* W = nullptr;
  int rc = single_setup(ctx, prob, phi, p, &W);
  if (rc) return rc;
  SlotHost& sl = W->slots[0];
  cudaStream_t s = ctx->stream;
  const size_t N = (size_t)prob->nx * prob->ny;
  // The solver's own stencil kernel at iteration 0 with beta = 0 and z = p: it forms
  // p_new = z + 0 * p_old = p in its window (the set-up zeroed p_old), q = M L^2 p_new and the
  // per-tile p.q partials, through the same tensor-copy or plain-load window path as in a solve.
  BX_CUDA(cudaMemcpyAsync(sl.d.z, p, 4 * N, cudaMemcpyDeviceToDevice, s));
  BX_CUDA(cudaMemsetAsync(sl.d.z_lo, 0, 4 * N, s));
  const int it0 = 0, on = 1;
  const double zero = 0.0;
  char* dsc = reinterpret_cast<char*>(W->d_sc);
  BX_CUDA(cudaMemcpyAsync(dsc + offsetof(SlotScalars, it), &it0, sizeof(int), cudaMemcpyHostToDevice, s));
  BX_CUDA(cudaMemcpyAsync(dsc + offsetof(SlotScalars, active), &on, sizeof(int), cudaMemcpyHostToDevice, s));
  BX_CUDA(cudaMemcpyAsync(dsc + offsetof(SlotScalars, beta), &zero, sizeof(double), cudaMemcpyHostToDevice, s));
  const LaunchCfg sc = cfg_of(ctx, W, 4);
  timed(ctx, EXT_KERNEL_STENCIL, [&] { launch_stencil(sc, W->aniso, W->sten_ty, ctx->d_err); });
  BX_CUDA(cudaGetLastError());
  BX_CUDA(cudaMemcpyAsync(q, sl.d.q, 4 * N, cudaMemcpyDeviceToDevice, s));
  std::vector<double> part((size_t)((prob->ny + 15) / 16) * ((prob->nx + kStTileX - 1) / kStTileX));
  BX_CUDA(cudaMemcpyAsync(part.data(), sl.d.pq_part, 8 * part.size(), cudaMemcpyDeviceToHost, s));
  BX_CUDA(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  BX_CUDA(cudaStreamSynchronize(s));
  if (*ctx->h_err) {
    BX_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
    BX_CUDA(cudaStreamSynchronize(s));
    g_last_error = "a bounded device wait (stencil tensor copy) ran out";
    return EXT_ETIMEOUT;
  }
  if (sum_pq) {
    double acc = 0.0;
    for (double v : part) acc += v;
    *sum_pq = acc;
  }
  return EXT_OK;
}

int ext_rhs(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f, double* b) {
  if (!ctx || !b) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  Workspace* W = nullptr;
  int rc = single_setup(ctx, prob, phi, f, &W);
  if (rc) return rc;
  const size_t N = (size_t)prob->nx * prob->ny;
  BX_CUDA(cudaMemcpyAsync(b, W->slots[0].d.b, 8 * N, cudaMemcpyDefault, ctx->stream));
  BX_CUDA(cudaStreamSynchronize(ctx->stream));
  return EXT_OK;
}

int ext_apply_preconditioner(ext_ctx* ctx, const ext_problem* prob, const float* phi,
                             const float* r, float* z, double* scale) {
  if (!ctx || !r || !z) return EXT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->api_mu);
  Workspace* W = nullptr;
  int rc = single_setup(ctx, prob, phi, r, &W);
  if (rc) return rc;
  SlotHost& sl = W->slots[0];
  const size_t N = (size_t)prob->nx * prob->ny;
  BX_CUDA(cudaMemcpyAsync(sl.d.r, r, 4 * N, cudaMemcpyDefault, ctx->stream));
  BX_CUDA(cudaMemsetAsync(sl.d.r_lo, 0, 4 * N, ctx->stream));
  BX_CUDA(cudaMemsetAsync(sl.d.q, 0, 4 * N, ctx->stream));
  BX_CUDA(cudaMemsetAsync(sl.d.q_lo, 0, 4 * N, ctx->stream));
  launch_prec(ctx, W, 2);
  BX_CUDA(cudaGetLastError());
  BX_CUDA(cudaMemcpyAsync(z, sl.d.z, 4 * N, cudaMemcpyDefault, ctx->stream));
  BX_CUDA(cudaStreamSynchronize(ctx->stream));
  if (scale) {
    const double a = 1.0 / (prob->hx * prob->hx), c = 1.0 / (prob->hy * prob->hy);
    const double m = std::max(a, c);
    *scale = (double)sl.d.wnorm * m * m;
  }
  return EXT_OK;
}

}  // extern "C"


// ---------------------------------------------------------------------------------------------
// Serving: continuous batching of independent extension requests.
//
// A worker thread owns its own stream and a fixed table of max_slots slots.  Between blocks of
// G iterations it (1) admits queued requests while the HBM footprint of the admitted slots
// stays within the budget, runs their set-up and first preconditioner pass, (2) replays the
// iteration graph over every slot that is still iterating (new and old together), and (3)
// retires slots whose solve has a final status: output kernel, copy-out for host buffers,
// result record, arena back to a size-keyed pool.  Work lists live in fixed device buffers
// that are rewritten when slots join or leave, so one captured graph serves every mix.
// ---------------------------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  ext_problem prob{};
  const float* phi = nullptr;
  const float* f = nullptr;
  float* out = nullptr;
  bool host_io = false;
  int status = EXT_PENDING;
  ext_result res{};
  Clock::time_point t_submit, t_admit;
};

struct ServeSlot {
  bool used = false;
  Req* req = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct ext_ctx::Serve {
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  bool stop = false;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_ticket = 1;
  int in_flight = 0;
  int worker_error = EXT_OK;
  Workspace* W = nullptr;       // capacity-sized slot table, work lists and graph
  std::vector<ServeSlot> slots;
  std::multimap<size_t, char*> pool;  // free arenas by size
  size_t budget = 0, used = 0;
  int cap_items = 0;
  WorkItem *d_new = nullptr, *d_ret = nullptr;
  int* d_aux = nullptr;          // [0] new stencil items, [1] retiring vector items
  int* h_aux = nullptr;
};

static int serve_alloc_lists(ext_ctx::Serve* S, int cap) {
  Workspace* W = S->W;
  cudaFree(W->d_st);
  cudaFree(W->d_sten);
  cudaFree(W->d_vec);
  cudaFree(W->d_gm);
  cudaFree(W->d_l1);
  cudaFree(W->d_l3);
  cudaFree(W->d_fold);
  cudaFree(W->d_unfold);
  cudaFree(W->d_tcl);
  cudaFree(W->d_prep);
  cudaFree(S->d_new);
  cudaFree(S->d_ret);
  W->d_st = W->d_sten = W->d_vec = W->d_gm = W->d_l1 = W->d_l3 = S->d_new = S->d_ret = nullptr;
  W->d_fold = W->d_unfold = W->d_tcl = W->d_prep = nullptr;
  BX_CUDA(cudaMalloc(&W->d_prep, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_fold, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_unfold, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_tcl, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_st, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_sten, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_l1, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_l3, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_vec, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&W->d_gm, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&S->d_new, sizeof(WorkItem) * cap));
  BX_CUDA(cudaMalloc(&S->d_ret, sizeof(WorkItem) * cap));
  S->cap_items = cap;
  // grids sized for the capacity
  W->n_st = W->n_vec = W->n_gm = W->n_sten = W->n_l1 = W->n_l3 = cap;
  W->n_fold = W->n_unfold = W->n_tcl = W->n_prep = cap;
  if (W->graph) {
    cudaGraphExecDestroy(W->graph);
    W->graph = nullptr;
  }
  return EXT_OK;
}

static int serve_init(ext_ctx* ctx) {
  std::unique_ptr<ext_ctx::Serve> S(new ext_ctx::Serve());
  const int cap = ctx->opt.max_slots;
  S->slots.resize(cap);
  Workspace* W = new Workspace();
  S->W = W;
  W->slots.resize(cap);
  BX_CUDA(cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking));
  BX_CUDA(cudaMalloc(&W->d_slots, sizeof(SlotDesc) * cap));
  BX_CUDA(cudaMalloc(&W->d_tcp, sizeof(SlotDesc) * kMirClasses * cap));
  BX_CUDA(cudaMalloc(&W->d_sc, sizeof(SlotScalars) * cap));
  BX_CUDA(cudaMemset(W->d_sc, 0, sizeof(SlotScalars) * cap));
  BX_CUDA(cudaMallocHost(&W->h_sc, sizeof(SlotScalars) * cap));
  memset(W->h_sc, 0, sizeof(SlotScalars) * cap);
  BX_CUDA(cudaMalloc(&W->d_counts, 11 * sizeof(int)));
  BX_CUDA(cudaMemset(W->d_counts, 0, 11 * sizeof(int)));
  BX_CUDA(cudaMalloc(&W->d_sl, sizeof(WorkItem) * cap));
  W->n_sl = cap;  // the per-slot grid is sized for the slot table
  BX_CUDA(cudaMalloc(&W->d_phis, sizeof(void*) * cap));
  BX_CUDA(cudaMalloc(&W->d_fs, sizeof(void*) * cap));
  BX_CUDA(cudaMalloc(&W->d_outs, sizeof(void*) * cap));
  BX_CUDA(cudaMalloc(&W->d_dirs, sizeof(int) * cap));
  BX_CUDA(cudaMallocHost(&W->h_ptrs, (3 * sizeof(void*) + sizeof(int)) * cap));
  BX_CUDA(cudaMalloc(&S->d_aux, 2 * sizeof(int)));
  BX_CUDA(cudaMallocHost(&S->h_aux, 2 * sizeof(int)));
  int rc = serve_alloc_lists(S.get(), 1 << 16);
  if (rc) return rc;
  size_t fr = 0, tot = 0;
  BX_CUDA(cudaMemGetInfo(&fr, &tot));
  S->budget = ctx->opt.hbm_budget ? ctx->opt.hbm_budget : fr / 2;
  ctx->serve = S.release();
  return EXT_OK;
}

// Rewrite the device work lists from the slots in use (in slot order).
static int serve_rebuild_lists(ext_ctx* ctx) {
  ext_ctx::Serve* S = ctx->serve;
  Workspace* W = S->W;
  std::vector<WorkItem> st, vec, gm, sl, l1, l3, fold, unfold, tcl, prep;
  bool aniso = false;
  for (int i = 0; i < (int)S->slots.size(); ++i) {
    if (!S->slots[i].used) continue;
    const SlotHost& h = W->slots[i];
    const SlotDesc& d = h.d;
    aniso |= d.aniso != 0;
    for (int t = 0; t < d.n_st_tiles; ++t) st.push_back({i, t});
    for (int t = 0; t < d.n_vec_items; ++t) vec.push_back({i, t});
    tc_items(h, i, gm, l1, l3, tcl);
    for (int t = 0; t < d.n_fold_items; ++t) fold.push_back({i, t});
    for (int t = 0; t < d.n_unfold_tiles; ++t) unfold.push_back({i, t});
    if (ctx->tc && !d.mir)
      for (int t = 0; t < d.n_prep_items; ++t) prep.push_back({i, t});
    sl.push_back({i, 0});
  }
  longest_first_tc(gm, W->slots);
  size_t need = 0;
  for (const auto* v : {&st, &vec, &gm, &l1, &l3, &fold, &unfold, &tcl, &prep}) need = std::max(need, v->size());
  if ((int)need > S->cap_items) {
    int cap = S->cap_items;
    while (cap < (int)need) cap *= 2;
    BX_CUDA(cudaStreamSynchronize(W->stream));
    int rc = serve_alloc_lists(S, cap);
    if (rc) return rc;
  }
  if (aniso != W->aniso && W->graph) {
    cudaGraphExecDestroy(W->graph);
    W->graph = nullptr;
  }
  W->aniso = aniso;
  cudaStream_t s = W->stream;
  auto put = [&](WorkItem* dst, const std::vector<WorkItem>& v) -> int {
    if (!v.empty()) BX_CUDA(cudaMemcpyAsync(dst, v.data(), sizeof(WorkItem) * v.size(), cudaMemcpyHostToDevice, s));
    return EXT_OK;
  };
  int rc = put(W->d_st, st);
  // the serving table keeps the 64 x 32 stencil tiles: its stencil list is the grid-tile list
  if (!rc) rc = put(W->d_sten, st);
  if (!rc) rc = put(W->d_vec, vec);
  if (!rc) rc = put(W->d_gm, gm);
  if (!rc) rc = put(W->d_sl, sl);
  if (!rc) rc = put(W->d_l1, l1);
  if (!rc) rc = put(W->d_l3, l3);
  if (!rc) rc = put(W->d_fold, fold);
  if (!rc) rc = put(W->d_unfold, unfold);
  if (!rc) rc = put(W->d_tcl, tcl);
  if (!rc) rc = put(W->d_prep, prep);
  if (rc) return rc;
  int counts[11] = {(int)st.size(), (int)vec.size(), (int)gm.size(), (int)sl.size(), (int)st.size(),
                    (int)l1.size(), (int)l3.size(), (int)fold.size(), (int)unfold.size(), (int)tcl.size(),
                    (int)prep.size()};
  BX_CUDA(cudaMemcpyAsync(W->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, s));
  // the host vectors die here: the copies above must finish first (pageable sources are staged)
  BX_CUDA(cudaStreamSynchronize(s));
  return EXT_OK;
}

static void finish_req(ext_ctx::Serve* S, Req* r, int status) {
  r->status = status;
  S->in_flight -= 1;
  S->cv_done.notify_all();
}

// Admit queued requests into free slots while the footprint fits; returns admitted slot indices.
static std::vector<int> serve_admit(ext_ctx* ctx) {
  ext_ctx::Serve* S = ctx->serve;
  std::vector<int> admitted;
  while (!S->queue.empty()) {
    int free_slot = -1;
    for (int i = 0; i < (int)S->slots.size(); ++i)
      if (!S->slots[i].used) {
        free_slot = i;
        break;
      }
    if (free_slot < 0) break;
    Req* r = S->queue.front();
    SlotHost probe;
    int rc = build_slot(ctx, r->prob, r->host_io, probe, nullptr, true);
    if (rc) {
      S->queue.pop_front();
      finish_req(S, r, rc);
      continue;
    }
    if (probe.bytes > S->budget) {
      S->queue.pop_front();
      finish_req(S, r, EXT_EADMIT);
      continue;
    }
    if (S->used + probe.bytes > S->budget) break;  // wait for running solves to free memory
    S->queue.pop_front();
    S->slots[free_slot].used = true;
    S->slots[free_slot].req = r;
    S->slots[free_slot].bytes = probe.bytes;
    S->used += probe.bytes;
    r->t_admit = Clock::now();
    admitted.push_back(free_slot);
  }
  return admitted;
}

static int serve_setup_slots(ext_ctx* ctx, const std::vector<int>& admitted) {
  ext_ctx::Serve* S = ctx->serve;
  Workspace* W = S->W;
  cudaStream_t s = W->stream;
  const int cap = (int)S->slots.size();
  const float** h_phis = (const float**)W->h_ptrs;
  const float** h_fs = h_phis + cap;
  float** h_outs = (float**)(h_fs + cap);
  int* h_dirs = (int*)(h_outs + cap);
  std::vector<WorkItem> fresh;
  for (int i : admitted) {
    Req* r = S->slots[i].req;
    SlotHost& sl = W->slots[i];
    char* arena = nullptr;
    auto it = S->pool.find(S->slots[i].bytes);
    if (it != S->pool.end()) {
      arena = it->second;
      S->pool.erase(it);
    }
    int rc = build_slot(ctx, r->prob, r->host_io, sl, arena);
    if (rc) return rc;
    set_slot_scalars(sl, W->d_sc + i);
    const size_t N = (size_t)r->prob.nx * r->prob.ny;
    if (r->host_io) {
      BX_CUDA(cudaMemcpyAsync(sl.phi_stage, r->phi, 4 * N, cudaMemcpyHostToDevice, s));
      BX_CUDA(cudaMemcpyAsync(sl.f_stage, r->f, 4 * N, cudaMemcpyHostToDevice, s));
      h_phis[i] = sl.phi_stage;
      h_fs[i] = sl.f_stage;
      h_outs[i] = sl.out_stage;
    } else {
      h_phis[i] = r->phi;
      h_fs[i] = r->f;
      h_outs[i] = r->out;
    }
    h_dirs[i] = r->prob.dir;
    BX_CUDA(cudaMemcpyAsync(W->d_phis + i, &h_phis[i], sizeof(void*), cudaMemcpyHostToDevice, s));
    BX_CUDA(cudaMemcpyAsync(W->d_fs + i, &h_fs[i], sizeof(void*), cudaMemcpyHostToDevice, s));
    BX_CUDA(cudaMemcpyAsync(W->d_outs + i, &h_outs[i], sizeof(void*), cudaMemcpyHostToDevice, s));
    BX_CUDA(cudaMemcpyAsync(W->d_dirs + i, &h_dirs[i], sizeof(int), cudaMemcpyHostToDevice, s));
    BX_CUDA(cudaMemcpyAsync(W->d_slots + i, &sl.d, sizeof(SlotDesc), cudaMemcpyHostToDevice, s));
    BX_CUDA(cudaMemcpyAsync(W->d_tcp + kMirClasses * i, sl.tcp, sizeof(SlotDesc) * kMirClasses,
                            cudaMemcpyHostToDevice, s));
    SlotScalars& sc = W->h_sc[i];
    memset(&sc, 0, sizeof(sc));
    sc.rtol2 = ctx->opt.rtol * ctx->opt.rtol;
    sc.maxit = ctx->opt.maxit > 0 ? ctx->opt.maxit : 10 * std::max(r->prob.nx, r->prob.ny);
    sc.fold_every = ctx->opt.true_res_every;
    sc.delta2 = ctx->opt.replace_factor * ctx->opt.replace_factor;
    sc.flexible = ctx->opt.flexible;
    sc.status = ST_RUNNING;
    BX_CUDA(cudaMemcpyAsync(W->d_sc + i, &sc, sizeof(SlotScalars), cudaMemcpyHostToDevice, s));
    for (int t = 0; t < sl.d.n_st_tiles; ++t) fresh.push_back({i, t});
  }
  int rc = serve_rebuild_lists(ctx);
  if (rc) return rc;
  // set-up of the new slots only, then their first preconditioner pass (need_prec gates it)
  BX_CUDA(cudaMemcpyAsync(S->d_new, fresh.data(), sizeof(WorkItem) * fresh.size(), cudaMemcpyHostToDevice, s));
  S->h_aux[0] = (int)fresh.size();
  BX_CUDA(cudaMemcpyAsync(S->d_aux, S->h_aux, sizeof(int), cudaMemcpyHostToDevice, s));
  LaunchCfg c;
  c.slots = W->d_slots;
  c.items = S->d_new;
  c.n_items = S->d_aux;
  c.grid = std::max(1, std::min((int)fresh.size(), ctx->sm_count * 8));
  c.stream = s;
  timed(ctx, EXT_KERNEL_SETUP, [&] { launch_setup(c, W->d_phis, W->d_fs, W->d_dirs); }, s);
  timed(ctx, EXT_KERNEL_SETUP, [&] { launch_rhs_scale(c); }, s);
  launch_prec(ctx, W, 1);
  BX_CUDA(cudaGetLastError());
  BX_CUDA(cudaStreamSynchronize(s));  // `fresh` is a pageable source
  return EXT_OK;
}

static int serve_retire(ext_ctx* ctx, const std::vector<int>& done) {
  ext_ctx::Serve* S = ctx->serve;
  Workspace* W = S->W;
  cudaStream_t s = W->stream;
  std::vector<WorkItem> ret;
  for (int i : done)
    for (int t = 0; t < W->slots[i].d.n_vec_items; ++t) ret.push_back({i, t});
  BX_CUDA(cudaMemcpyAsync(S->d_ret, ret.data(), sizeof(WorkItem) * ret.size(), cudaMemcpyHostToDevice, s));
  S->h_aux[1] = (int)ret.size();
  BX_CUDA(cudaMemcpyAsync(S->d_aux + 1, S->h_aux + 1, sizeof(int), cudaMemcpyHostToDevice, s));
  LaunchCfg c;
  c.slots = W->d_slots;
  c.items = S->d_ret;
  c.n_items = S->d_aux + 1;
  c.grid = std::max(1, std::min((int)ret.size(), ctx->sm_count * 8));
  c.stream = s;
  timed(ctx, EXT_KERNEL_OUTPUT, [&] { launch_output(c, W->d_fs, W->d_outs); }, s);
  for (int i : done) {
    Req* r = S->slots[i].req;
    if (r->host_io) {
      const size_t N = (size_t)r->prob.nx * r->prob.ny;
      BX_CUDA(cudaMemcpyAsync(r->out, W->slots[i].out_stage, 4 * N, cudaMemcpyDeviceToHost, s));
    }
  }
  BX_CUDA(cudaStreamSynchronize(s));
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  for (int i : done) {
    Req* r = S->slots[i].req;
    const SlotScalars& sc = W->h_sc[i];
    const int st = map_status(sc.status, sc.n_known, r->prob);
    r->res.status = st;
    r->res.iters = sc.it;
    r->res.relres_true = sc.bb > 0 ? std::sqrt(sc.rr_true / sc.bb) : 0.0;
    r->res.relres_rec = sc.bb > 0 ? std::sqrt(sc.rr / sc.bb) : 0.0;
    r->res.n_known = sc.n_known;
    r->res.n_unknown = r->prob.nx * r->prob.ny - sc.n_known;
    r->res.ms_queue = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
    r->res.ms_solve = std::chrono::duration<double, std::milli>(now - r->t_admit).count();
    r->res.err_est = err_estimate(sc);
    S->pool.emplace(S->slots[i].bytes, W->slots[i].arena);
    W->slots[i].arena = nullptr;
    S->used -= S->slots[i].bytes;
    S->slots[i] = ServeSlot{};
    finish_req(S, r, st);
  }
  return EXT_OK;
}

static void serve_fail_all(ext_ctx* ctx, int rc) {
  ext_ctx::Serve* S = ctx->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  S->worker_error = rc;
  for (auto& sl : S->slots)
    if (sl.used) {
      finish_req(S, sl.req, rc);
      sl = ServeSlot{};
    }
  while (!S->queue.empty()) {
    finish_req(S, S->queue.front(), rc);
    S->queue.pop_front();
  }
}

static void serve_loop(ext_ctx* ctx) {
  ext_ctx::Serve* S = ctx->serve;
  Workspace* W = S->W;
  cudaSetDevice(ctx->device);
  for (;;) {
    std::vector<int> admitted;
    int active = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (auto& sl : S->slots) active += sl.used ? 1 : 0;
      S->cv.wait(lk, [&] { return S->stop || !S->queue.empty() || active > 0; });
      if (S->stop && S->queue.empty() && active == 0) return;
      admitted = serve_admit(ctx);
      active += (int)admitted.size();
    }
    int rc = EXT_OK;
    if (!admitted.empty()) rc = serve_setup_slots(ctx, admitted);
    if (!rc && active > 0) {
      rc = ensure_graph(ctx, W);
      if (!rc) {
        if (cudaGraphLaunch(W->graph, W->stream) != cudaSuccess) rc = EXT_ECUDA;
        ctx->launches += W->graph_nodes;
      }
    }
    if (!rc) {
      const int cap = (int)S->slots.size();
      if (cudaMemcpyAsync(W->h_sc, W->d_sc, sizeof(SlotScalars) * cap, cudaMemcpyDeviceToHost, W->stream) != cudaSuccess ||
          cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, W->stream) != cudaSuccess ||
          cudaStreamSynchronize(W->stream) != cudaSuccess)
        rc = EXT_ECUDA;
      else if (*ctx->h_err)
        rc = EXT_ETIMEOUT;
    }
    if (!rc) {
      std::vector<int> done;
      for (int i = 0; i < (int)S->slots.size(); ++i)
        if (S->slots[i].used && W->h_sc[i].status != ST_RUNNING) done.push_back(i);
      if (!done.empty()) {
        rc = serve_retire(ctx, done);
        if (!rc) rc = serve_rebuild_lists(ctx);
      }
    }
    if (rc) {
      cudaGetLastError();
      serve_fail_all(ctx, rc);
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) return;
    }
  }
}

extern "C" {

int ext_submit(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f, float* out,
               uint64_t* ticket) {
  if (!ctx || !prob || !phi || !f || !out || !ticket) return EXT_EINVAL;
  int rc = validate_problem(prob);
  if (rc) return rc;
  const bool dev = is_device_ptr(phi) && is_device_ptr(f) && is_device_ptr(out);
  const bool host = !is_device_ptr(phi) && !is_device_ptr(f) && !is_device_ptr(out);
  if (!dev && !host) return EXT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (!ctx->serve) {
      rc = serve_init(ctx);
      if (rc) return rc;
      ctx->serve->worker = std::thread(serve_loop, ctx);
    }
  }
  ext_ctx::Serve* S = ctx->serve;
  Req* r = new Req();
  r->prob = *prob;
  r->phi = phi;
  r->f = f;
  r->out = out;
  r->host_io = host;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->worker_error) {
      delete r;
      return S->worker_error;
    }
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
    S->in_flight += 1;
    *ticket = r->ticket;
  }
  S->cv.notify_all();
  return EXT_OK;
}

int ext_poll(ext_ctx* ctx, uint64_t ticket, ext_result* res) {
  if (!ctx) return EXT_EINVAL;
  if (!ctx->serve) return EXT_ENOTFOUND;
  ext_ctx::Serve* S = ctx->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return EXT_ENOTFOUND;
  Req* r = it->second;
  if (r->status == EXT_PENDING) return EXT_PENDING;
  const int st = r->status;
  if (res) *res = r->res;
  S->reqs.erase(it);
  delete r;
  return st;
}

int ext_drain(ext_ctx* ctx) {
  if (!ctx) return EXT_EINVAL;
  if (!ctx->serve) return EXT_OK;
  ext_ctx::Serve* S = ctx->serve;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] { return S->in_flight == 0; });
  return S->worker_error;
}

void ext_serve_shutdown(ext_ctx* ctx) {
  if (!ctx || !ctx->serve) return;
  ext_ctx::Serve* S = ctx->serve;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  Workspace* W = S->W;
  cudaStreamSynchronize(W->stream);
  for (auto& kv : S->pool) cudaFree(kv.second);
  for (auto& sl : W->slots) cudaFree(sl.arena);
  W->slots.clear();
  cudaStream_t st = W->stream;
  free_workspace(W);
  cudaStreamDestroy(st);
  cudaFree(S->d_new);
  cudaFree(S->d_ret);
  cudaFree(S->d_aux);
  cudaFreeHost(S->h_aux);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
  ctx->serve = nullptr;
}

}  // extern "C"
