// Operator apply without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the operator: host
// applications that reserve the whole device-memory budget up front and forbid libraries from
// taking more (a simulation code that owns its memory pool, or a process sharing the GPU under a
// fixed quota), and hot loops in which a cudaMalloc/cudaFree pair would synchronise the device and
// stall every other stream.  For them, ext_apply_biharmonic_noalloc computes the same
// q = M L^2 p as ext_apply_biharmonic with every byte of scratch (slot descriptor, known-node
// mask, per-tile partial sums) taken from one file-scope device array of fixed size, and without
// creating a context.
//
// Limits and sharing: grids of at most kNoAllocMaxNodes nodes and kNoAllocMaxTiles stencil tiles.
// The array exists once per device that loads the library and lives until the process exits.
// All calls on a device share it and it keeps the previous call's contents; every byte a call
// reads is written earlier in that same call, so nothing has to start at zero.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on the array and must
// be serialised by the caller.  The array's device address is looked up once per device, by the
// first call made with that device current; the cached address does not survive cudaDeviceReset
// (the module is loaded anew).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/biharm_ext.h"
#include "common.cuh"
#include "kernels.h"

namespace bx {

constexpr size_t kNoAllocBytes = size_t(1) << 21;          // 2 MiB per device
constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 20;     // 1024 x 1024
constexpr int kNoAllocMaxTiles = 32768;
constexpr size_t kOffDesc = 0;
constexpr size_t kOffSum = 1024;                           // one double: p.q
constexpr size_t kOffPart = 2048;                          // kNoAllocMaxTiles doubles
constexpr size_t kOffMask = kOffPart + 8 * kNoAllocMaxTiles;
static_assert(sizeof(SlotDesc) <= kOffSum, "descriptor does not fit its scratch slot");
static_assert(kOffMask + kNoAllocMaxNodes <= kNoAllocBytes, "scratch array too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Known-node mask from sign(phi) into the scratch (1 = unknown), same rule as the set-up kernel.
__global__ void k_noalloc_mask(const float* __restrict__ phi, int n, int extend_out,
                               uint8_t* __restrict__ mask) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float ph = phi[e];
    const bool known = extend_out ? (ph < 0.f) : (ph > 0.f);
    mask[e] = known ? 0 : 1;
  }
}

// One block: sum of the per-tile partials in index order (thread-strided, fixed tree).
__global__ void __launch_bounds__(256) k_noalloc_sum(const double* __restrict__ part, int n,
                                                     double* __restrict__ out) {
  __shared__ double red[64];
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) a += part[t];
  block_sum2<256>(a, b, red);
  if (threadIdx.x == 0) *out = a;
}

}  // namespace bx

using namespace bx;

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};
thread_local std::string g_noalloc_err;
}  // namespace

extern "C" const char* ext_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" int ext_apply_biharmonic_noalloc(const ext_problem* prob, const float* phi,
                                            const float* p, float* q, double* sum_pq,
                                            void* cuda_stream) {
  if (!prob || !phi || !p || !q) return EXT_EINVAL;
  if (validate_problem(prob) != EXT_OK) {
    g_noalloc_err = "invalid problem (sizes below 4 or above 2^30 nodes, spacing not finite and "
                    "positive, unknown boundary rule or direction)";
    return EXT_EINVAL;
  }
  const int64_t n = (int64_t)prob->nx * prob->ny;
  const int64_t tiles = ((int64_t)prob->nx + kStTileX - 1) / kStTileX *
                        (((int64_t)prob->ny + kStTileY - 1) / kStTileY);
  if (n > kNoAllocMaxNodes || tiles > kNoAllocMaxTiles) {
    g_noalloc_err = "grid too large for the fixed no-allocation scratch (at most 1048576 nodes "
                    "and 32768 stencil tiles of 64x32)";
    return EXT_EINVAL;
  }
  // the kernels dereference phi, p and q: device (or managed) memory only
  if (!is_device_ptr(phi) || !is_device_ptr(p) || !is_device_ptr(q)) {
    g_noalloc_err = "phi, p and q must be device pointers";
    return EXT_EINVAL;
  }
  // Once per device, with that device current: the device address of the scratch array.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    g_noalloc_err = "no usable current CUDA device";
    return EXT_ECUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        g_noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return EXT_ECUDA;
      }
      g_noalloc_ptr[dev] = ptr;
    }
    base = g_noalloc_ptr[dev];
  }
  unsigned char* scratch = static_cast<unsigned char*>(base);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  SlotDesc d{};
  d.nx = prob->nx;
  d.ny = prob->ny;
  d.bcx = prob->bc_x;
  d.bcy = prob->bc_y;
  d.n_st_tiles = (int)tiles;
  set_weights(d, prob->hx, prob->hy);
  d.mask = reinterpret_cast<uint8_t*>(scratch + kOffMask);
  double* part = reinterpret_cast<double*>(scratch + kOffPart);
  double* sum = reinterpret_cast<double*>(scratch + kOffSum);
  SlotDesc* d_desc = reinterpret_cast<SlotDesc*>(scratch + kOffDesc);

  cudaError_t e = cudaMemcpyAsync(d_desc, &d, sizeof(SlotDesc), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const int nn = (int)n;
    int grid = (nn + 255) / 256;
    grid = grid < 4096 ? grid : 4096;
    k_noalloc_mask<<<grid, 256, 0, s>>>(phi, nn, prob->dir == EXT_EXTEND_OUT ? 1 : 0, d.mask);
    launch_apply(d_desc, (int)tiles, d.aniso != 0, p, q, part, s);
    k_noalloc_sum<<<1, 256, 0, s>>>(part, (int)tiles, sum);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && sum_pq) e = cudaMemcpyAsync(sum_pq, sum, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_noalloc_err = std::string("CUDA: ") + cudaGetErrorString(e);
    return EXT_ECUDA;
  }
  return EXT_OK;
}
