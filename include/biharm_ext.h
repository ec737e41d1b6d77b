/*
 * biharm_ext.h -- C ABI of the GB300 biharmonic field extension library (libbiharm_ext.so).
 *
 * The library extends a field f, known on the part Omega of a rectangular grid picked by the sign
 * of a level set function phi, to the whole grid by solving the masked discrete biharmonic
 * equation (Moroney, Lusmore, McCue, McElwain, "Extending fields in a level set method by solving
 * a biharmonic equation", arXiv 1704.08897):
 *
 *   - Sec. 2.1, eq. (discrete_biharmonic): at every unknown node the 13-point stencil
 *     20 f_ij - 8 (edge neighbours) + 2 (diagonals) + (nodes at distance 2) = 0, with the values
 *     at known nodes acting as data; stencils at the domain edge use ghost nodes set by the
 *     boundary rule of each axis.
 *   - Sec. 2.2, Algorithm 1: the system is solved by conjugate gradients with the fast Poisson
 *     solve on the whole rectangle (zero-augmentation of D\Omega into D, separable transforms,
 *     division by the squared eigenvalue sums) as the preconditioner.
 *
 * Layout: every grid array is row-major [ny][nx] (x contiguous), float32.
 * Pointers: phi, f and out may be device pointers or host pointers (pageable or pinned); host
 * arrays are copied in and out on the context's stream inside the call.
 * Ownership: the caller owns phi, f and out and keeps them alive until ext_solve / ext_solve_batch
 * returns, or until ext_poll reports a final status for a submitted request.  The library owns
 * every workspace, transform plan and CG state.  out may alias f.
 * Errors: every entry point returns EXT_OK (0), EXT_PENDING (1) or a negative EXT_E* code;
 * ext_strerror() names it.  No entry point aborts the process or traps on the GPU.
 */
#ifndef BIHARM_EXT_H
#define BIHARM_EXT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary rule of one axis.  SYMMETRIC is the Neumann case of Example 1 (half-sample reflection,
 * cosine transform); PERIODIC wraps around (Examples 2 and 4, Fourier transform); DIRICHLET is
 * Algorithm 1's padding (f = 0 and lap f = 0 on the boundary, sine transform). */
typedef enum { EXT_BC_SYMMETRIC = 0, EXT_BC_PERIODIC = 1, EXT_BC_DIRICHLET = 2 } ext_bc;

/* Fig. 1: extend out = field known inside the interface (phi < 0); extend in = field known
 * outside (phi > 0).  phi == 0 is an unknown node in both directions. */
typedef enum { EXT_EXTEND_OUT = 0, EXT_EXTEND_IN = 1 } ext_dir;

/* Arithmetic of the iteration.  In every mode the CG inner products are FP64, the iterate x is
 * updated in FP64 every iteration, and the recursive residual is replaced by the FP64 true
 * residual b - A x whenever it has fallen by replace_factor since the last replacement, at
 * least every true_res_every iterations, and before convergence is declared.
 *   FP32        : FP32 vectors, compensated FP32 stencil, FP32 CUDA-core transform products.
 *   MIXED_FP16  : as FP32, transforms on the tcgen05 tensor cores: every operand as four exact
 *                 8-bit integer slices per 128-wide exponent block, stored as FP16, products
 *                 summed exactly per slice order in FP32 accumulators.
 *   MIXED_BF16  : the same slices stored as BF16 (results identical to MIXED_FP16).
 * The iteration runs on 2^e b with e chosen from ||b||; the answer is scaled back exactly.    */
typedef enum {
  EXT_PREC_FP32 = 1,
  EXT_PREC_MIXED_BF16 = 2,
  EXT_PREC_MIXED_FP16 = 3
} ext_prec;

typedef struct {
  int32_t nx, ny;      /* grid nodes along x (contiguous) and y; each >= 4                     */
  double hx, hy;       /* node spacings (> 0); only hx/hy matters, the solution is scale-free  */
  int32_t bc_x, bc_y;  /* ext_bc of each axis                                                  */
  int32_t dir;         /* ext_dir                                                              */
} ext_problem;

typedef struct {
  int32_t prec;            /* ext_prec; default EXT_PREC_FP32                                  */
  double rtol;             /* relative residual target ||b - A x|| / ||b||; default 1e-8       */
  int32_t maxit;           /* iteration cap; 0 = 10 * max(nx, ny)                              */
  int32_t true_res_every;  /* longest run of iterations between residual replacements; 200     */
  double replace_factor;   /* replace once ||r|| < replace_factor * ||r at last replacement||;
                              default 1e-2                                                     */
  int32_t iters_per_launch;/* CG iterations per CUDA-graph replay; default 10                 */
  size_t hbm_budget;       /* bytes the serving queue may hold for admitted requests; 0 = 50%
                              of free device memory at ext_create                             */
  int32_t flexible;        /* 1 = flexible (Polak-Ribiere) beta, 0 = Fletcher-Reeves beta;
                              default 0: on the benchmark grids it takes fewer iterations and
                              ends nearer the exact solution at the same residual              */
  int32_t max_slots;       /* serving: most requests in flight at once; default 256            */
  int32_t profile;         /* 1: launch every kernel directly (no CUDA graphs) and time each one
                              with CUDA events on the context stream (ext_profile_read); 0    */
  int32_t autotune;        /* 1: the stencil's tile height (16 or 32 rows of 64 nodes) is chosen
                              per workspace shape by timing both on the first solve, and kept in
                              a process-wide table and, if the environment variable
                              EXT_TUNE_CACHE names a file, in that file; 0: tile_y; default 1.
                              Results do not depend on the tile.                              */
  int32_t tile_y;          /* the stencil's tile height when autotune = 0: 16 or 32 (default) */
  int32_t low_modes;       /* mixed modes: 1 = the lowest 32 x 32 modes of each transform
                              problem (those with the largest weights) come from six-slice
                              tensor-core products of about 48 bits instead of the four-slice
                              stages: 20-28% fewer iterations at more cost per iteration;
                              0 = all modes from the four-slice stages; 2 = on for grids with a
                              side of at least 2048 nodes and for every grid of an ext_solve /
                              ext_solve_batch / ext_solve_multi call whose grids hold at least
                              2048^2 nodes together, off otherwise (default; served requests
                              take the per-grid rule).  With 2, a grid's iterates therefore
                              depend on the call it is solved in; 0 or 1 fix them.            */
  int64_t wait_cycles;     /* bound, in SM clock cycles, of every wait of a kernel for its own
                              tensor copies and tensor-core pipeline; a wait that runs out makes
                              the kernel drain what it issued and return, and the call returns
                              EXT_ETIMEOUT; 0 = 4e9 (about two seconds)                       */
  int32_t fold;            /* mixed modes: 1 = an axis whose two mirror classes (ceil(n/2) nodes
                              each), padded to 128, fit in the axis padded to 128 runs its
                              transforms per class (even and odd vectors under i -> n-1-i: half
                              the products per stage) (default); 0 = full-size transforms      */
} ext_options;

/* Kernel kinds reported by ext_profile_read. */
enum {
  EXT_KERNEL_SETUP = 0,          /* mask, right-hand side, CG state                          */
  EXT_KERNEL_STENCIL = 1,        /* p = z + beta p, q = M L^2 p, p.q                         */
  EXT_KERNEL_UPDATE = 2,         /* x += alpha p, r -= alpha q, r.r                          */
  EXT_KERNEL_TRUE_RESIDUAL = 3,  /* FP64 b - A x and residual replacement                    */
  EXT_KERNEL_PREC0 = 4,          /* transform stages 0..3 of the fast Poisson preconditioner */
  EXT_KERNEL_PREC1 = 5,
  EXT_KERNEL_PREC2 = 6,
  EXT_KERNEL_PREC3 = 7,
  EXT_KERNEL_OUTPUT = 8,         /* out = f on Omega, x elsewhere                            */
  EXT_KERNEL_SPLIT = 9,          /* residual -> 16-bit integer slices (mixed modes, unfolded)  */
  EXT_KERNEL_PREC_FINISH = 10,   /* per-slot r.z, z.q -> rho, beta                            */
  EXT_KERNEL_PQ_FINISH = 11,     /* per-slot p.q -> alpha                                     */
  EXT_KERNEL_LOW_FWD = 12,       /* low-mode correction: forward product, middle, inverse    */
  EXT_KERNEL_LOW_MID = 13,
  EXT_KERNEL_LOW_INV = 14,
  EXT_KERNEL_UNFOLD = 15,        /* mirror classes -> masked z, r.z, z.q (folded slots)       */
  EXT_KERNEL_FOLD = 16,          /* residual -> mirror classes' slices (folded slots)          */
  EXT_KERNEL_KINDS = 17
};

/* A three-dimensional problem (Sec. 3 Example 2: the equations of Sec. 2 in three dimensions;
 * at an interior node with equal spacings the operator is the 25-point squared 7-point
 * Laplacian).  Grid arrays are row-major [nz][ny][nx] (x contiguous), float32. */
typedef struct {
  int32_t nx, ny, nz;        /* nodes along x (contiguous), y and z; each >= 4                 */
  double hx, hy, hz;         /* node spacings (> 0); the solution depends only on their ratios */
  int32_t bc_x, bc_y, bc_z;  /* ext_bc of each axis                                            */
  int32_t dir;               /* ext_dir                                                        */
} ext_problem3;

typedef struct {
  int32_t status;      /* EXT_OK, EXT_ENOTCONV, EXT_EBREAKDOWN, ...                            */
  int32_t iters;       /* CG iterations taken                                                  */
  double relres_true;  /* FP64 ||b - A x|| / ||b|| of the returned x, recomputed on the GPU     */
  double relres_rec;   /* the recursively updated residual at exit                            */
  int32_t n_unknown;   /* |D \ Omega|                                                          */
  int32_t n_known;     /* |Omega|                                                              */
  double ms_queue;     /* serving: submit -> admission                                         */
  double ms_solve;     /* admission (or call start) -> result written                          */
  double err_est;      /* estimated relative A-norm error ||x* - x||_A / ||x*||_A of the returned
                          iterate: CG's step terms alpha_j rho_j (rho = r.z) of the last 8
                          iterations over their sum over all iterations (the Hestenes-Stiefel
                          estimate with a delay of 8; 0 when no iteration ran)                 */
} ext_result;

enum {
  EXT_OK = 0,
  EXT_PENDING = 1,
  EXT_EINVAL = -1,      /* bad size, spacing, enum, null pointer or NaN in phi                 */
  EXT_ENOKNOWN = -2,    /* no known node and no Dirichlet axis: solution not unique           */
  EXT_ENOMEM = -3,      /* device allocation failed                                            */
  EXT_EADMIT = -4,      /* request footprint exceeds the serving HBM budget                    */
  EXT_ENOTCONV = -5,    /* maxit reached; out holds the best iterate                           */
  EXT_EBREAKDOWN = -6,  /* p.Ap <= 0 or a non-finite scalar in CG                              */
  EXT_ETIMEOUT = -7,    /* a bounded device wait ran out                                       */
  EXT_ECUDA = -8,       /* a CUDA runtime call failed                                          */
  EXT_ENOTSUP = -9,     /* mode not available on this device                                   */
  EXT_ENOTFOUND = -10   /* unknown serving ticket                                              */
};

typedef struct ext_ctx ext_ctx;

/* Fill *opt with the defaults listed above. */
void ext_options_default(ext_options* opt);

/* Create a context bound to the current CUDA device and to cuda_stream (a cudaStream_t; NULL =
 * a stream the context creates).  opt may be NULL (defaults).  Returns EXT_ENOTSUP when the
 * mixed modes are requested on a device without tcgen05 (compute capability 10.x). */
int ext_create(const ext_options* opt, void* cuda_stream, ext_ctx** out);

/* One extension (Sec. 2.1 problem, Algorithm 1 solve): out = f at known nodes (bit copy),
 * the PCG solution at unknown nodes.  Blocks until the result is in out.  res may be NULL. */
int ext_solve(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f,
              float* out, ext_result* res);

/* count independent extensions of possibly different sizes solved together: every CG stage is
 * one launch over all still-iterating problems, iterations are replayed from CUDA graphs.
 * Each result equals what ext_solve gives for that problem alone, within the stated tolerance. */
int ext_solve_batch(ext_ctx* ctx, int count, const ext_problem* probs, const float* const* phi,
                    const float* const* f, float* const* out, ext_result* results);

/* Several fields known on the same Omega (one phi, e.g. the components of a velocity field, as in
 * the level-set application of Sec. 5 of the paper, where each step extends more than one field):
 * f[i] and out[i], i < count, are the fields and their extensions; phi, the problem and the
 * transform plans are shared and the fields iterate together in the same launches.  Each result
 * equals ext_solve of that field alone.  Pointers as for ext_solve_batch. */
int ext_solve_multi(ext_ctx* ctx, const ext_problem* prob, const float* phi, int count,
                    const float* const* f, float* const* out, ext_result* results);

/* Serving: enqueue one request (returns at once with a ticket).  A device-resident loop admits
 * queued requests as slots and HBM free up (continuous batching: new requests join the
 * iterations of those already running).  Thread-safe. */
int ext_submit(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f,
               float* out, uint64_t* ticket);

/* EXT_PENDING while the request is queued or running, else its final status (and *res). */
int ext_poll(ext_ctx* ctx, uint64_t ticket, ext_result* res);

/* Block until every submitted request has finished. */
int ext_drain(ext_ctx* ctx);

/* Release every resource of the context (waits for in-flight work). */
void ext_destroy(ext_ctx* ctx);

const char* ext_strerror(int code);

/* Accumulated CUDA-event time (ms) and launch count of each kernel kind since the last reset,
 * recorded only by contexts created with profile = 1.  Arrays hold `kinds` entries; either may be
 * NULL.  reset != 0 clears the totals after reading. */
int ext_profile_read(ext_ctx* ctx, int kinds, double* total_ms, int64_t* launches, int reset);

/* Number of kernels this context has launched (graph replays count every kernel node). */
int64_t ext_launch_count(ext_ctx* ctx);

/* Stencil tile (x by y nodes) of the workspace the context's last solve used. */
int ext_stencil_tile(ext_ctx* ctx, int32_t* tile_x, int32_t* tile_y);

/* Text of the last CUDA or allocation failure seen by the calling thread ("" if none). */
const char* ext_last_error(void);

/* ---- single stages of the path, for verification (device pointers, [ny][nx] float32) ---- */

/* As ext_solve, but writes the FP64 iterate (device pointer): out64 = f at known nodes, x at
 * unknown nodes, so a caller can recompute ||b - A x|| / ||b|| exactly (the FP32 out of
 * ext_solve cannot carry a relative residual of 1e-8 for this ill-conditioned operator). */
int ext_solve_f64(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f,
                  double* out64, ext_result* res);

/* q = M L^2 p on the full grid (eq. discrete_biharmonic with the boundary rules), M zeroing the
 * known nodes picked by phi; p must be zero at known nodes for this to be A p (Algorithm 1,
 * matvec).  Runs the solver's own stencil kernel as at iteration 0 with beta = 0 and z = p, so q
 * is bit for bit what a solve computes for that direction.  phi, p and q are device pointers
 * (host pointers return EXT_EINVAL).  sum_pq (host, may be NULL) receives the dot p.q (FP64 sum
 * of the kernel's compensated per-tile partials). */
int ext_apply_biharmonic(ext_ctx* ctx, const ext_problem* prob, const float* phi,
                         const float* p, float* q, double* sum_pq);

/* b = -M L^2 (f at known nodes, zero elsewhere), in FP64 (Algorithm 1, right-hand side). */
int ext_rhs(ext_ctx* ctx, const ext_problem* prob, const float* phi, const float* f, double* b);

/* z = M (L^2)^+ M r on the full grid with the context's precision (Algorithm 1, fast_poisson,
 * pseudo-inverse when both axes are symmetric/periodic); r must be zero at known nodes.
 * The result is scale-free: z is (L^2)^+ r times a positive constant reported in *scale
 * (may be NULL), since CG does not depend on the preconditioner's scale. */
int ext_apply_preconditioner(ext_ctx* ctx, const ext_problem* prob, const float* phi,
                             const float* r, float* z, double* scale);

/* Transform basis of one axis, computed on the host (no GPU, no context): the dense orthonormal
 * eigenvector matrix of the axis's 1-D negative second difference T (h = 1) that the fast Poisson
 * preconditioner applies (Algorithm 1: sine transform for Dirichlet edges; Example 1: cosine
 * transform, DCT-II, for symmetric edges; Example 2: real Fourier basis for periodic edges), and
 * its eigenvalues.  Q (n*n doubles, row-major: Q[i*n + k] is the k-th eigenvector at node i) and
 * lam (n doubles, lam[k] its eigenvalue) are caller-owned host arrays; T = Q diag(lam) Q^T.
 * Returns EXT_OK, or EXT_EINVAL for n < 4, n > 32768, an unknown bc or a NULL array. */
int ext_axis_basis(int32_t n, ext_bc bc, double* Q, double* lam);

/* Three-dimensional extension (Sec. 3 Example 2).  Solves the masked biharmonic system on the
 * nz x ny x nx box by preconditioned CG from x = 0 to the context's rtol (relative FP64 residual on
 * the unknowns), the preconditioner being the fast Poisson solve on the box by separable
 * transforms along the three axes.  It runs the CUDA-core double-float path in every precision
 * mode (double-float CG vectors, compensated products in the transforms, FP64 right-hand side and
 * residual replacements), one problem per call, the iteration driven from the host.  phi, f and
 * out are device pointers ([nz][ny][nx] float32; host pointers return EXT_EINVAL); out = f at
 * known nodes (bit copy), the extension elsewhere; out may alias f.  res (may be NULL) receives
 * status, iterations, the true and recursive relative residuals, counts and err_est.  Returns
 * EXT_OK, EXT_EINVAL (sizes, spacings, enums, NaN phi, a non-finite known value, host pointers),
 * EXT_ENOKNOWN, EXT_ENOMEM, EXT_ENOTCONV (out holds the last iterate), EXT_EBREAKDOWN or
 * EXT_ECUDA.  Allocates its workspace per call (about 90 bytes per node). */
int ext_solve3d(ext_ctx* ctx, const ext_problem3* prob, const float* phi, const float* f, float* out,
                ext_result* res);

/* q = M L^2 M p for the 3-D problem (the solver's operator passes; M zeroes known nodes), with
 * the spacings normalised so that the largest 1/h^2 is 1.  phi, p, q: device pointers
 * [nz][ny][nx]; q receives the hi plane of the double-float result (exact for integer p of
 * moderate size). */
int ext_apply_biharmonic3d(ext_ctx* ctx, const ext_problem3* prob, const float* phi, const float* p,
                           float* q);

/* z = M (L^2)^+ M r for the 3-D problem (the solver's preconditioner; pseudo-inverse when no axis
 * is Dirichlet), scale-free: z is (L^2)^+ M r times the positive constant written to *scale (may
 * be NULL).  phi, r, z: device pointers [nz][ny][nx]; z receives the hi plane. */
int ext_apply_preconditioner3d(ext_ctx* ctx, const ext_problem3* prob, const float* phi, const float* r,
                               float* z, double* scale);

/* One mirror class of the same axis, computed on the host (no GPU, no context); this is what the
 * tensor-core preconditioner applies on axes where folding halves the work (Sec. 2.2: the fast
 * transforms' even/odd symmetry).  The mirror i -> n-1-i maps T onto itself, and the axis has an
 * orthonormal eigenbasis of even and odd vectors: the DCT-II and DST-I bases as they are, and for
 * the periodic rule the real Fourier basis sampled at i + 1/2 (same eigenspaces as
 * ext_axis_basis's).  With h = ceil(n/2), Q (h*h doubles, row-major) holds the class's vectors
 * restricted to nodes 0..h-1, in ascending order of eigenvalue, and lam (h doubles) their
 * eigenvalues; columns beyond the class's mode count are zero (eigenvalue 0), and for odd n the
 * odd class's row h-1 (the middle node) is zero.  cls: 0 = even, 1 = odd.  For r on the n nodes,
 * the class transform of the folded vector (r[i] + r[n-1-i], or r[i] alone at the middle node, for
 * cls 0; r[i] - r[n-1-i] for cls 1) equals the full transform's class coefficients.  Returns
 * EXT_OK, or EXT_EINVAL for n < 4, n > 32768, an unknown bc or cls, or a NULL array. */
int ext_axis_class_basis(int32_t n, ext_bc bc, int32_t cls, double* Q, double* lam);

/* The tensor-core operand form of the same basis, computed on the host (no GPU, no context): Q
 * and Q^T, zero-padded to np x np (np = n rounded up to a multiple of 128), each row cut into
 * blocks of 128 columns and each block with exponent E into four exact integer slices,
 * v = c0 2^(E-8) + c1 2^(E-16) + c2 2^(E-24) + c3 2^(E-32) + (rest below 2^(E-33)), |c0| <= 255,
 * |c1|, |c2|, |c3| <= 128.  codes (caller-owned, 8 np^2 words): [Q slices 0..3][Q^T slices 0..3],
 * each slice an [np][np] row-major plane of the integers c_k as FP16 (type 0) or BF16 (type 1)
 * bit patterns; exps (caller-owned, 2 np^2/128 bytes): [Q rows][Q^T rows], each [np][np/128].
 * Returns EXT_OK, or EXT_EINVAL for n < 4, n > 32768, an unknown bc or type, or a NULL array. */
int ext_axis_slices(int32_t n, ext_bc bc, int32_t type, uint16_t* codes, int8_t* exps);

/* ---- operator apply that allocates nothing ----
 *
 * Same result as ext_apply_biharmonic (q = M L^2 p, and the FP64 sum p.q into *sum_pq, which may
 * be NULL), for callers that cannot allocate device memory when they need it: host applications
 * that reserve the whole device-memory budget up front and forbid libraries from taking more, and
 * latency-critical loops in which cudaMalloc/cudaFree would synchronise the device.  The paper has
 * no counterpart; this is a property of the library, not of the method.
 * No context is needed.  phi, p and q are device pointers, [ny][nx] float32 (host pointers return
 * EXT_EINVAL); the call runs on cuda_stream (NULL = the legacy default stream) and returns after
 * that stream has finished its work.
 * Scratch: one fixed 2 MiB array per device (grids up to 1,048,576 nodes and 32,768 stencil
 * tiles of 64x32; larger grids return EXT_EINVAL, see ext_noalloc_last_error).  The first call on
 * a device looks up that array's device address (a lookup that allocates nothing).  The looked-up
 * address is kept for the life of the process and does not survive cudaDeviceReset.  All calls on a device share the array: calls whose GPU work
 * overlaps race and must be serialised by the caller.  Nothing in it needs to start at zero. */
int ext_apply_biharmonic_noalloc(const ext_problem* prob, const float* phi, const float* p,
                                 float* q, double* sum_pq, void* cuda_stream);

/* Reason for the last EXT_EINVAL / EXT_ECUDA of ext_apply_biharmonic_noalloc in this thread. */
const char* ext_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BIHARM_EXT_H */
