/*
 * helm.h - C ABI of libhelm: CNN-preconditioned flexible GMRES for the 2D
 * heterogeneous Helmholtz equation with a PML, on NVIDIA B300 (sm_103a).
 *
 * Problem (eq. 1 with the sign flipped, eq. 3):  -Lap u - (omega / c(x))^2 u = f
 * on an nx x ny interior grid of spacing h surrounded by `width` PML cells per
 * side.  The PML damping is quadratic in the depth into the layer (eq. 2) and
 * enters as the complex coordinate stretch s = 1 + i sigma / omega; the discrete
 * operator is the complex-symmetric 5-point stencil
 *
 *   (A u)_{j,i} = -[ a_{i+1/2}(u_{i+1}-u_i) - a_{i-1/2}(u_i-u_{i-1})
 *                  + b_{j+1/2}(u_{j+1}-u_j) - b_{j-1/2}(u_j-u_{j-1}) ] / h^2
 *                 - s_x(i) s_y(j) k^2 u_{j,i},
 *   a_{i+1/2} = s_y(j) / s_x(i+1/2),  b_{j+1/2} = s_x(i) / s_y(j+1/2),
 *
 * with zero values outside the grid.  A = A^T exactly.
 *
 * Conventions shared by every call:
 *  - Grid of a system: Nx = nx + 2 width, Ny = ny + 2 width, n = Nx * Ny points,
 *    row-major [Ny][Nx] (x fastest).
 *  - A "batch vector" holds nrhs right-hand sides for every system of a
 *    context: for system s = 0..nsys-1 in order, nrhs blocks of n_s points.
 *    Complex values are interleaved (re, im): HELM_C64 = 2 x float (8 B),
 *    HELM_C128 = 2 x double (16 B).  Pointers must be 16-byte aligned.
 *  - Every array argument is caller-owned DEVICE memory unless marked host.
 *    The library owns only its context, network and workspace allocations.
 *  - Every call is asynchronous on the caller's stream (`stream` is a
 *    cudaStream_t passed as void*; NULL = legacy default stream), except
 *    helm_fgmres_solve and helm_train_step, which synchronise that stream
 *    before they return because they hand back host-side results.
 *  - Errors: no call aborts, traps or exits.  Each returns a helm_status;
 *    helm_last_error() gives a message for the calling thread.  Invalid
 *    arguments are detected on the host before anything is launched.
 *  - Columns: a call on nrhs right-hand sides works on nsys * nrhs columns;
 *    more than HELM_MAX_COLUMNS (one CUDA grid dimension) is rejected with
 *    HELM_ERR_INVALID_ARG.
 *  - Environment switches: HELM_DISABLE_GRAPHS=1 runs the
 *    BF16 network eagerly instead of replaying captured CUDA graphs;
 *    HELM_AUTOTUNE=0 keeps the first rows-per-tile variant of every row-tile
 *    convolution and the first tile shape of the FP32 stencil instead of timing
 *    the variants on first use; HELM_DISABLE_TC=1
 *    runs the BF16 convolutions on CUDA cores, HELM_DISABLE_ROW=1 the narrow
 *    layers on the 9-box tcgen05 kernels (comparison and testing aids).  The first
 *    two are read once per process, the last two when a network is created.  None
 *    changes a result beyond FP32 summation order, and the first two none at all.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HELM_API __attribute__((visibility("default")))
#else
#define HELM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_ctx helm_ctx;    /* grids, coefficients, workspace */
typedef struct helm_unet helm_unet;  /* network weights (FP64 master + BF16 copy), AdamW state */

typedef enum {
  HELM_OK = 0,
  HELM_ERR_INVALID_ARG = 1,
  HELM_ERR_CUDA = 2,
  HELM_ERR_OOM = 3,
  HELM_NOT_CONVERGED = 4, /* iteration budget spent before the tolerance was met */
  HELM_BREAKDOWN = 5,     /* Z rank-deficient: h_{j+1,j} or R_jj vanished before convergence */
  HELM_NAN = 6,           /* a NaN/Inf appeared in a norm or Hessenberg entry */
  HELM_TIMEOUT = 7        /* a device-side wait ran out of its iteration budget */
} helm_status;

typedef enum { HELM_C64 = 0, HELM_C128 = 1 } helm_dtype;

#define HELM_MAX_COLUMNS 65535

typedef struct {
  int nx, ny;  /* interior cells */
  double h;    /* grid spacing (same unit as c / omega) */
} helm_grid;

typedef struct {
  int width;         /* PML cells per side (0 = none) */
  double sigma_max;  /* damping at the outermost node; <= 0 selects 2 omega (Tab. 1: 2 at omega = 1) */
} helm_pml;

/* CGS2: classical Gram-Schmidt, two passes per iteration (4 sweeps over the basis).
 * DCGS2: the same two passes with the second one delayed into the next iteration, where it shares
 * the sweep of the first pass (2 sweeps over the basis); the preconditioner then sees each basis
 * vector after its first pass (admissible in flexible GMRES, eq. 4). */
typedef enum { HELM_ORTH_CGS2 = 0, HELM_ORTH_DCGS2 = 1 } helm_orth;

typedef struct {
  int m;            /* Krylov dimension per cycle (Alg. 1), 1..HELM_MAX_M */
  int max_restarts; /* cycles per inner solve (plain path: total cycles) */
  int max_outer;    /* FP64 refinement steps (mixed path) */
  double tol;       /* stop when the FP64 true ||b - A x|| / ||b|| <= tol (eq. 10) */
  double inner_tol; /* mixed path: relative reduction asked of each FP32 inner solve */
  int mixed;        /* 0: plain FP64 (C128 vectors, FP64 network); 1: FP32 Krylov + BF16 network + FP64 refinement */
  int orth;         /* helm_orth */
} helm_solve_opts;

#define HELM_MAX_M 4096

typedef struct {
  int iters;           /* preconditioned Krylov iterations spent on this column */
  int restarts;        /* cycles */
  int outer;           /* FP64 refinement steps */
  double relres_true;  /* final FP64 ||b - A x|| / ||b|| */
  double relres_est;   /* last Givens estimate, relative to ||b|| */
  helm_status status;  /* HELM_OK, HELM_NOT_CONVERGED, HELM_BREAKDOWN or HELM_NAN */
} helm_solve_info;

/* ---- context ---------------------------------------------------------- */

/* Set up nsys systems (a1: k^2 = (omega/c)^2 and the 1-D PML stretch profiles, eq. 2).
 * grid[nsys], pml[nsys], omega[nsys]: host arrays, one entry per system
 * (systems may differ in size: an uneven batch).  c_dev: device array of all
 * systems' velocities concatenated, each [Ny][Nx], real, in FP64 when
 * c_is_fp64 != 0 else FP32; read during this call only (stream-ordered).
 * c must be > 0 and finite (checked on the device; HELM_ERR_INVALID_ARG). */
HELM_API helm_status helm_create(helm_ctx** out, int nsys, const helm_grid* grid, const helm_pml* pml,
                        const double* omega, const void* c_dev, int c_is_fp64, void* stream);
HELM_API helm_status helm_destroy(helm_ctx* ctx);
/* Replace the velocities of every system of ctx (grids, PMLs and frequencies unchanged), e.g. the next
 * batch of a training set: k^2 and c / 1500 m/s are recomputed on `stream`.  c_dev as in helm_create;
 * c must be > 0 and finite (HELM_ERR_INVALID_ARG; the previous values are then partly overwritten).
 * Synchronises `stream`. */
HELM_API helm_status helm_set_velocity(helm_ctx* ctx, const void* c_dev, int c_is_fp64, void* stream);
/* Total points of one batch vector per right-hand side (sum of n_s), and the system count. */
HELM_API int64_t helm_points(const helm_ctx* ctx);
HELM_API int helm_num_systems(const helm_ctx* ctx);

/* ---- operator (a2) ---------------------------------------------------- */

/* y = A x for a batch vector of nrhs right-hand sides per system.  x and y must not overlap. */
HELM_API helm_status helm_apply(helm_ctx* ctx, const void* x, void* y, helm_dtype dtype, int nrhs, void* stream);
/* y = A^H x (= conj(A conj(x)) since A = A^T); used by the loss gradient (eq. 9). */
HELM_API helm_status helm_apply_adjoint(helm_ctx* ctx, const void* x, void* y, helm_dtype dtype, int nrhs, void* stream);
/* y = A_F x: the paper's own discretisation (Sec. 2.1, Tab. 1), Fourier differentiation on the
 * periodic grid that includes the PML, with the stretched derivatives of the same PML (eq. 2):
 *   A_F u = -[ (1/s_x) D_x((1/s_x) D_x u) + (1/s_y) D_y((1/s_y) D_y u) ] - k^2 u,
 *   D u = IDFT(i kappa DFT(u)) along one axis, kappa_q = 2 pi q / (N h), the Nyquist mode set to zero,
 * s = 1 + i sigma / omega at the grid nodes.  An alternative to helm_apply (the 5-point operator);
 * the solver and the network use helm_apply's operator.  Every system's Nx and Ny must be powers of
 * two in [16, 1024] (HELM_ERR_INVALID_ARG otherwise).  x, y: batch vectors that must not overlap. */
HELM_API helm_status helm_apply_fourier(helm_ctx* ctx, const void* x, void* y, helm_dtype dtype, int nrhs,
                                        void* stream);
/* out_host[col] = ||b - A x|| / ||b|| in FP64 for every column (eq. 10); x, b are C128. Synchronises. */
HELM_API helm_status helm_relres(helm_ctx* ctx, const void* x, const void* b, int nrhs, double* out_host, void* stream);

/* ---- neural operator (a3) ---------------------------------------------- */

/* Network layout (Sec. 3.1, Fig. 2, read as): 4 levels of widths 16/32/64/128, two 3x3 convs
 * (pad 1, bias, ReLU) per level, 2x2 max-pool down, 2x2 stride-2 transposed conv up (bias, no
 * activation), decoder input concat[skip, up], final 1x1 conv 16 -> 2.  Inputs
 * (Re v, Im v, c / 1500 m/s); outputs (Re z, Im z).
 * weights_host: nweights = helm_unet_param_count() doubles, per layer weight then bias, layers in
 * the order enc1a enc1b enc2a enc2b enc3a enc3b bota botb up3 dec3a dec3b up2 dec2a dec2b up1
 * dec1a dec1b final; conv weights [Cout][Cin][kh][kw], transposed-conv weights [Cin][Cout][2][2]. */
HELM_API size_t helm_unet_param_count(void);
/* Layer l (0..17): writes c_in, c_out, kind (0 = 3x3 conv, 1 = 2x2 up-conv, 2 = 1x1 conv). */
HELM_API helm_status helm_unet_layer(int l, int* c_in, int* c_out, int* kind);
HELM_API helm_status helm_unet_create(helm_unet** out, const double* weights_host, size_t nweights);
/* Network kinds: 0 = the network above (helm_unet_create); 1 = the paper's own variant (Sec. 3.1, Tab. 2,
 * read as): inputs (Re v, Im v, c / 1500 m/s, Re sigma_c, Im sigma_c) with the complex PML field
 * sigma_c = s_x s_y - 1 (eq. 2); encoder of four 8x8 stride-2 pad-3 convolutions (5 -> 32 -> 32 -> 32
 * -> 32 channels), decoder of four 8x8 stride-2 pad-3 transposed convolutions (32 -> 32, then 64 -> 32
 * on [decoder, skip] concatenations), PReLU (one slope per layer) after each, batch normalisation folded
 * into the convolutions, final 1x1 conv 32 -> 2; grid zero-padded to multiples of 16.
 * Weights of kind 1 (665,930 doubles): per layer weight, bias, PReLU slope (none for the output layer);
 * layers enc1 enc2 enc3 enc4 dec3 dec2 dec1 dec0 out; conv weights [Cout][Cin][8][8], transposed-conv
 * weights [Cin][Cout][8][8], output weights [2][32].  Kind 1 serves helm_precond_apply and
 * helm_fgmres_solve (BF16 on tcgen05 tensor cores, or FP64 on CUDA cores) and helm_train_step /
 * helm_loss_grad (C64 batches: forward on the tcgen05 layers in BF16 with FP32 accumulation, the
 * pre-activations kept in BF16, backward on CUDA cores in FP32; C128: FP64 on CUDA cores). */
HELM_API size_t helm_unet_param_count_kind(int kind);
HELM_API helm_status helm_unet_create_kind(helm_unet** out, int kind, const double* weights_host, size_t nweights);
HELM_API helm_status helm_unet_destroy(helm_unet* net);
/* Copy the FP64 master weights back to the host (after training). */
HELM_API helm_status helm_unet_get_weights(const helm_unet* net, double* weights_host, size_t nweights);
/* Replace the weights (same layout as helm_unet_create) from caller-owned DEVICE memory, FP64, e.g.
 * a parameter tensor updated by an outside optimiser; the BF16 / FP32 / FP64 working copies are
 * rebuilt on `stream` before the call returns control to the stream's later work.  The AdamW state
 * of helm_train_step is left as it is.  HELM_ERR_INVALID_ARG on a NULL pointer or a wrong count;
 * non-finite values are not checked (the next solve reports HELM_NAN). */
HELM_API helm_status helm_unet_set_weights(helm_unet* net, const double* weights_dev, size_t nweights, void* stream);

/* z = h^2 N_theta(alpha v, c) / alpha per column, alpha = sqrt(n) / ||v|| (eq. 6): the network sees a
 * unit-RMS input and approximates the inverse of the dimensionless operator h^2 A.  dtype HELM_C64:
 * BF16 network with FP32 accumulation (3x3 and up-convs on tcgen05 tensor cores); HELM_C128: FP64
 * network on CUDA cores.  v, z batch vectors; a zero column gives z = 0 (network kind 1, HELM_C64:
 * such columns are skipped by every layer, which is how the solver leaves converged columns out).
 * HELM_C64 runs: the second call for the same (network, system, nrhs) captures the network's launch
 * sequence into a CUDA graph that later calls replay on the library's own stream (ordered after and
 * before the caller's stream by events); the first call that meets a new row-tile conv layer shape
 * times its tile variants once, which synchronises the caller's stream that one time. */
HELM_API helm_status helm_precond_apply(helm_ctx* ctx, const helm_unet* net, const void* v, void* z,
                               helm_dtype dtype, int nrhs, void* stream);

/* ---- solver (a4-a8) ---------------------------------------------------- */

/* Solve A x = b for nrhs right-hand sides per system by FGMRES (Alg. 1) with z_j = N_theta(v_j)
 * (net = NULL: z_j = v_j, i.e. GMRES).  b, x: C128 batch vectors; x holds x0 on entry and the
 * solution on exit (the best iterate when not converged).  opts: host.  info: host array of
 * nsys * nrhs entries (column = system-major, rhs-minor).  Returns HELM_OK when every column met
 * opts->tol, HELM_NOT_CONVERGED / HELM_BREAKDOWN / HELM_NAN when at least one did not. */
HELM_API helm_status helm_fgmres_solve(helm_ctx* ctx, const helm_unet* net, const void* b, void* x, int nrhs,
                              const helm_solve_opts* opts, helm_solve_info* info, void* stream);

/* Residual-estimate history of the last helm_fgmres_solve on this context: for column 0, the Givens
 * estimate |g_{j+1}| of every iteration scaled to ||b|| (relative to the true residual at the start
 * of its cycle).  Copies up to max_entries values to est_host (may be NULL); returns the count. */
HELM_API int helm_solve_history(const helm_ctx* ctx, double* est_host, int max_entries);

/* ---- training (a9) ------------------------------------------------------ */

/* One optimisation step of the physics-informed loss (eqs. 8-9) over a batch of one source per
 * system: b is a C64 batch vector with nrhs = 1.  Loss = mean_s ||b_s - A_s u_s||^2 / ||b_s||^2,
 * u_s = N_theta(alpha b_s, c_s) / alpha.  Gradient by the adjoint stencil and the conv backward
 * kernels; global-norm clip to `clip` (<= 0: none); AdamW (beta 0.9/0.999, eps 1e-8) with
 * learning rate lr and decoupled weight decay wd.  loss_host: host pointer for the batch loss
 * before the update (may be NULL).  grad_norm_host: the pre-clip gradient norm (may be NULL). */
HELM_API helm_status helm_train_step(helm_ctx* ctx, helm_unet* net, const void* b, double lr, double wd,
                            double clip, double* loss_host, double* grad_norm_host, void* stream);
/* AdamW state of helm_train_step, for checkpoints that resume training exactly: m_host and v_host
 * hold helm_unet_param_count() doubles each (first and second moments, weights_host layout) and
 * step the number of updates taken (bias correction).  get: zeros and 0 before the first step.
 * Both synchronise the device. */
HELM_API helm_status helm_unet_get_adam(const helm_unet* net, double* m_host, double* v_host, int64_t* step);
HELM_API helm_status helm_unet_set_adam(helm_unet* net, const double* m_host, const double* v_host, int64_t step);
/* Loss and its gradient only (no update): grad_dev receives helm_unet_param_count() doubles in the
 * weights_host layout.  dtype HELM_C64: b is C64 and the BF16 network path is differentiated (as in
 * helm_train_step); HELM_C128: b is C128 and the FP64 network path is differentiated. */
HELM_API helm_status helm_loss_grad(helm_ctx* ctx, const helm_unet* net, const void* b, helm_dtype dtype,
                                    double* loss_host, double* grad_dev, void* stream);

/* ---- allocation-free relative residual (the paper has no counterpart) ---------
 * For callers that must not allocate device memory during a call: e.g. a process whose device
 * memory is reserved up front by another framework's caching allocator, or a latency-critical
 * loop in which a cudaMalloc would synchronise the device.  Computes the same per-column
 * ||b - A x|| / ||b|| (FP64) as helm_relres, but writes it to DEVICE memory
 * relres_dev[nsys * nrhs] (column = system-major, rhs-minor), stores no residual vector, and
 * calls no cudaMalloc, cudaFree or allocating library routine.  x, b: C128 batch vectors.
 * Its per-block partial sums live in one fixed device array of 2^20 doubles (8 MiB) that every
 * GPU loading this library holds until the process exits; a batch needing more than that
 * (2 x ceil(Nx/128) x ceil(Ny/8) doubles per column, summed over columns) is rejected with
 * HELM_ERR_INVALID_ARG.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any stream
 * capture.  All calls share the array, which keeps the last call's contents (every partial is
 * written before it is read, so nothing needs clearing): calls that overlap on the GPU, on
 * different streams or threads, race on it.  Asynchronous on `stream`. */
HELM_API helm_status helm_relres_noalloc(helm_ctx* ctx, const void* x, const void* b, int nrhs, double* relres_dev,
                                         void* stream);

/* ---- measurement (no paper counterpart: instrumentation of the path above) ---- */

/* Phase timers of helm_fgmres_solve, measured with CUDA events on the solver's stream:
 * 0 preconditioner (U-Net), 1 stencil w = A z, 2 CGS2 orthogonalisation + norm, 3 Givens / back
 * substitution, 4 FP64 true residual + v1, 5 solution update.  Enabling (on != 0) resets the
 * accumulators; timing adds one event pair per phase and iteration. */
#define HELM_NUM_PHASES 6
HELM_API helm_status helm_profile_enable(helm_ctx* ctx, int on);
/* ms_host[HELM_NUM_PHASES]: accumulated milliseconds; counts_host (may be NULL): intervals timed. */
HELM_API helm_status helm_profile_read(const helm_ctx* ctx, double* ms_host, int64_t* counts_host);
/* work_host[HELM_NUM_PHASES]: algorithmic work issued in each phase since helm_profile_enable:
 * flops for phase 0 (70,816 per pixel and network application), bytes for the others (stencil
 * 16 B/pt + 4 B/pt of k^2; orthogonalisation 32 nv + 48 B/pt (CGS2) or 16 nv + 48 B/pt (DCGS2) per
 * iteration with nv basis vectors, counted for the columns active in that iteration). */
HELM_API helm_status helm_profile_work(const helm_ctx* ctx, double* work_host);
/* Kernels launched by this library in this process so far (all contexts). */
HELM_API uint64_t helm_launch_count(void);
/* Tile heights the autotuner chose so far for the row-tile convolutions (no counterpart in the
 * paper: the library picks, per layer shape, the fastest of a few rows-per-tile variants the first
 * time the shape runs).  Writes up to max_entries records of 6 ints {C_out, 8-channel input slices,
 * images, H, W, rows per tile} to out (host) and returns how many it wrote. */
HELM_API int helm_tuned_tiles(int* out, int max_entries);

/* ---- per-layer network application (test and diagnostic aid; no paper counterpart) ----------
 * One layer of the BF16 network exactly as helm_precond_apply runs it, on caller-owned NHWC BF16
 * device tensors, so that each tensor-core kernel can be checked against a plain convolution.
 *   layer: 0..16 in helm_unet_layer order (3x3 convs add the bias and apply ReLU; 2x2 up-convs
 *          add the bias), or HELM_LAYER_DEC1B_FINAL: the last 3x3 conv (16 -> 16, ReLU, BF16
 *          rounding) with the final 1x1 conv 16 -> 2 fused into its epilogue, written as FP32
 *          pairs out[B][H][W][2] (output scale 1).
 *   in0:   [B][H][W][C0] BF16; C0 = c_in, except the first layer (a 16-channel tensor of which
 *          channels 0..2 are read with nonzero weights) and the decoder's first convs (C0 = c_in / 2,
 *          the skip connection).  in1: the up-sampled half [B][H][W][c_in / 2] of a decoder conv's
 *          concatenated input, NULL for every other layer.
 *   out:   [B][H][W][c_out] BF16 ([B][2H][2W][c_out] for up-convs).
 *   variant: 0 = the kernel the preconditioner picks for this shape (row-tile kernels: the
 *          autotuned rows per tile); k >= 1 = the k-th rows-per-tile variant of the row-tile kernel;
 *          -1 = the 9-box tcgen05 kernel.  A variant the layer does not have: HELM_ERR_INVALID_ARG.
 *   ry_out: rows per tile of the row-tile kernel that ran (0 for the 9-box kernels); may be NULL.
 * Pointers 16-byte aligned; B, H, W >= 1.  Asynchronous on `stream`.  HELM_ERR_INVALID_ARG when
 * the tcgen05 path is unavailable on the current device. */
#define HELM_LAYER_DEC1B_FINAL 17

/* One layer of network kind 1 (the paper's variant, see helm_unet_create_kind) in the BF16 path,
 * exactly as helm_precond_apply runs it (tcgen05, BF16 operands, FP32 accumulation, bias and PReLU
 * in FP32, BF16 output), on caller-owned NHWC BF16 device tensors; a test and diagnostic aid with no
 * paper counterpart.  H x W is the layer's 5x5 GEMM grid: the output grid of an encoder layer, the
 * input grid of a decoder layer.
 *   layer 0:    enc1 (Tab. 2: 8x8, stride 2, pad 3, PReLU).  in0: the network input packed
 *               space-to-depth, [B][H][W][32], channel (2 (y % 2) + x % 2) * 8 + c holding input
 *               channel c (5 used of 8) of pixel (y, x) of the 2H x 2W grid.  out: [B][H][W][32].
 *   layer 1..3: enc2..enc4.  in0: the previous encoder output [B][2H][2W][32].  out: [B][H][W][32].
 *               Layers 0..2 with H and W even run in the phase form the preconditioner uses on its
 *               16-padded grids (a 3x3 convolution over 4 x 4 input blocks with the 2 x 2 output phases
 *               as 128 GEMM columns); layer 3 and odd grids in the 5x5 form.
 *   layer 4:    dec3 (8x8 transposed, stride 2, pad 3, PReLU).  in0: [B][H][W][32].  out: [B][2H][2W][32].
 *   layer 5..7: dec2..dec0 on the concatenation [in0, in1], both [B][H][W][32] (in1: the skip
 *               connection).  out: [B][2H][2W][32].
 *   HELM_PAPER_LAYER_DEC0_FINAL: dec0 with the output layer (1x1 conv 32 -> 2 on the BF16
 *               activation) fused into its epilogue, written as FP32 pairs out[B][2H][2W][2] (scale 1).
 * in1 must be NULL except for layers 5..7.  Pointers 16-byte aligned; B, H, W >= 1, B H W <= 2^29.
 * Asynchronous on `stream`; a pipeline timeout is reported by the next solve or by the network's
 * error check.  HELM_ERR_INVALID_ARG for another network kind or where the tcgen05 path is
 * unavailable. */
#define HELM_PAPER_LAYER_DEC0_FINAL 8
HELM_API helm_status helm_paper_layer_forward(const helm_unet* net, int layer, const void* in0, const void* in1,
                                              void* out, int B, int H, int W, void* stream);
HELM_API helm_status helm_unet_layer_forward(const helm_unet* net, int layer, int variant, const void* in0,
                                             const void* in1, void* out, int B, int H, int W, int* ry_out,
                                             void* stream);

/* ---- failure injection and pipeline-wait budget (test aids; no paper counterpart) -------------
 * Every pipeline wait of the TMA / tcgen05 kernels (FP32 stencil, tensor-core convolutions) gives
 * up after a budget of clock64 cycles.  The kernel then records an error code, stops issuing work,
 * lets the copies it already requested land (a bound of its own, about one second), waits for its
 * issued tensor-core operations, releases its tensor memory and returns.  helm_fgmres_solve checks
 * the recorded codes at the end of every cycle, before the solution update, and returns
 * HELM_TIMEOUT with x left at the last completed cycle's iterate.  These two calls let a test make
 * that happen without faulting the GPU.  Both settings are process-wide; while a fault is armed or
 * the budget differs from the default, the network runs without CUDA graphs. */
typedef enum {
  HELM_FAULT_NONE = 0,
  HELM_FAULT_STENCIL_TILE = 1, /* the FP32 TMA stencil requests no data for its first tile */
  HELM_FAULT_CONV_TILE = 2,    /* a tcgen05 convolution requests no data for its first tile */
  HELM_FAULT_ALLOC = 3         /* a workspace reservation fails with HELM_ERR_OOM (no cudaMalloc call) */
} helm_fault;
/* Budget of every pipeline wait launched from now on, in clock64 cycles; cycles <= 0 restores the
 * default (2e9, about one second at the B300's clock). */
HELM_API helm_status helm_set_wait_budget(int64_t cycles);
/* Arm `site` for its next `count` occurrences (launches, or workspace reservations); site
 * HELM_FAULT_NONE or count <= 0 disarms.  HELM_ERR_INVALID_ARG for an unknown site. */
HELM_API helm_status helm_inject_fault(int site, int count);

/* Tile shapes the autotuner chose so far for the FP32 TMA stencil (no counterpart in the paper: the
 * first call for a grid shape times a few tile heights and pipeline depths with CUDA events, which
 * synchronises the caller's stream that one time; every candidate gives bit-identical results).
 * Writes up to max_entries records of 6 ints {Nx, Ny, nrhs, adjoint, rows per tile, stages} and
 * returns how many it wrote. */
HELM_API int helm_tuned_stencil(int* out, int max_entries);
/* Test aid: run every later FP32 stencil launch with tile candidate `variant` (1: 32 rows x 2 stages,
 * 2: 16 x 4, 3: 32 x 3, 4: 64 x 2) instead of the tuned one; 0 restores tuning.  Process-wide. */
HELM_API helm_status helm_set_stencil_variant(int variant);

/* Thread-local message for the last non-OK status returned on this thread. */
HELM_API const char* helm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
