// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/biharm_ext.h"
#include "common.cuh"

namespace bx {

struct LaunchCfg {
  const SlotDesc* slots;   // device array of slot descriptors
  const SlotDesc* tcp = nullptr;  // tensor-core problems (kMirClasses per slot), mixed modes
  const WorkItem* items;   // device work list
  const int* n_items;      // device count of valid items (persistent kernels read it)
  int grid;
  cudaStream_t stream;
  long long wait_cycles = 0;  // bound of the kernels' pipeline waits (0: the default bound)
};

// host helpers (api.cu): stencil weights of (L_y (+) L_x)^2 for spacings hx, hy; the problem
// checks every entry point applies (EXT_OK or EXT_EINVAL); whether a pointer is device (or
// managed) memory that kernels may dereference
void set_weights(SlotDesc& d, double hx, double hy);
int validate_problem(const ext_problem* p);
bool is_device_ptr(const void* p);

// grid kernels (kernels_grid.cu)
void launch_setup(const LaunchCfg& c, const float* const* phis, const float* const* fs,
                  const int* dirs);
void launch_rhs_scale(const LaunchCfg& c);
// err receives 1 if a bounded wait for a tensor copy ran out; tile_y = 16 or 32 (tiles 64 wide)
void launch_stencil(const LaunchCfg& c, bool aniso, int tile_y, int* err);
int stencil_blocks_per_sm(int tile_y);
// shared-memory carveout of the stencil kernels (once per process and device)
cudaError_t stencil_init();
// per-slot p.q -> alpha (after the stencil)
void launch_pq_finish(const LaunchCfg& c);
void launch_update(const LaunchCfg& c);
void launch_true_residual(const LaunchCfg& c);
void launch_output(const LaunchCfg& c, const float* const* fs, float* const* outs);
void launch_output64(const SlotDesc* slot, int n, const float* f, double* out, cudaStream_t s);
// per-slot reduction of the last preconditioner stage's r.z, z.q partials -> rho, beta
void launch_prec_finish(const LaunchCfg& c, int mode);
void launch_apply(const SlotDesc* slot, int n_tiles, bool aniso, const float* p, float* q,
                  double* part, cudaStream_t s);

// fast Poisson preconditioner, FP32 CUDA-core transform products (kernels_gemm_simt.cu).
// stage 0..3 = forward x, forward y (+ eigenvalue weights), inverse x, inverse y (+ mask, dots).
// mode 0: slots with active iterations; mode 1: slots with a pending preconditioner pass;
// mode 2: every slot (verification entry point).
void launch_prec_simt(const LaunchCfg& c, int stage, int mode);
// the mirror classes' residuals of folded slots in double-float (c.slots = slots, c.tcp = the
// transform problems, items: the unfold tiles of 32 x 8 class nodes)
void launch_simt_fold(const LaunchCfg& c, int mode);

// tensor-core variant (kernels_gemm_tc.cu): exact block-scaled integer slice planes stored as
// FP16 (split_kind 0) or BF16 (split_kind 1); err receives 1 if a bounded wait ran out.
void launch_prec_tc(const LaunchCfg& c, int stage, int mode, int split_kind, int* err);
// residual -> integer slice planes of the first stage's A operand, slots with no folded axis
// (items of 32 rows x 128 columns)
void launch_prec_tc_prepare(const LaunchCfg& c, int mode, int split_kind);
int tc_planes(int split_kind);
// low-mode correction of the tensor-core preconditioner: kind 0 = forward product with the tiles'
// shares of G (one CTA per 128 rows of y), kind 1 = inverse product (one CTA per 128 rows of x,
// walking the y-tiles); the middle step one block per (problem, 128 rows of x)
void launch_low_tc(const LaunchCfg& c, int kind, int mode, int split_kind, int* err);
void launch_low_mid(const LaunchCfg& c, int mode, int split_kind);
// mirror fold: residual -> slices of each class's first operand (c.slots = slots, items of the
// folded slots), and class results -> masked z with the r.z, z.q partials
void launch_tc_fold(const LaunchCfg& c, int mode, int split_kind);
void launch_unfold(const LaunchCfg& c, int mode);
int tc_block();
bool tc_supported();

// Tensor-core preconditioner of the 3-D path (mixed modes, every side a multiple of 128): the
// residual slicing and the six transform products as launches of the 2-D kernels over prepared
// descriptors (one per launch, [0] = slicing, [1..6] = products), built by the context.
struct Tc3 {
  bool on = false;
  SlotDesc* d_descs = nullptr;
  const WorkItem* d_items[7] = {};
  const int* d_counts = nullptr;  // [7]
  int n_items[7] = {};
  int split = 0;
  int* d_err = nullptr;
  long long wait_cycles = 0;
  int sm_count = 148;
  double* part = nullptr;         // the last product's tile partials (4 doubles per tile)
  int n_tiles3 = 0;
  std::vector<void*> owned;       // device allocations, freed by the solve
};
// the solve's vectors the descriptors refer to
struct Tc3Io {
  const float *rh, *rl, *qh, *ql;
  float *zh, *zl;
  const uint8_t* mask;
};

// three-dimensional extension (solve3d.cu): the CUDA-core double-float path, host-driven CG
struct Solve3Args {
  int nx, ny, nz;
  int bc[3];               // ext_bc of x, y, z
  int dir;                 // ext_dir
  double h[3];             // spacings of x, y, z
  const float* q[3];       // per axis: Q and Q^T as double-float planes [2][np][np] (device)
  const float* qt[3];
  int np[3];
  const double* lam[3];    // per axis: eigenvalues of T (h = 1), n entries (host)
  double rtol;
  int maxit;
  int true_res_every;
  double replace_factor;
  cudaStream_t stream;
  long long* launches;     // incremented by every kernel launch (host counter)
  // builds the tensor-core preconditioner for the given vectors (empty: CUDA-core transforms)
  std::function<int(const Tc3Io&, Tc3&)> tc_build;
};
int solve3d_run(const Solve3Args& a, const float* phi, const float* f, float* out, ext_result* res,
                std::string* err);
int apply3d_operator(const Solve3Args& a, const float* phi, const float* p, float* q, std::string* err);
int apply3d_preconditioner(const Solve3Args& a, const float* phi, const float* r, float* z, double* scale,
                           std::string* err);
// opt the tensor-core kernels into their dynamic shared memory (once per process and device)
cudaError_t tc_init();

}  // namespace bx
