/*
 * sdx.h - C ABI of the GB300 library for the decoupled (interface-strain) Stokes operator of
 * Huber, Ruede, Waluga and Wohlmuth, "Highly sparse surface couplings for subdomain-wise
 * isoviscous Stokes finite element discretizations" (arXiv:1604.07994), and the all-at-once
 * Uzawa multigrid built on it.
 *
 * Discretisation (paper Sec. 4-5): unit cube, n^3 hexahedral cells each split into six Kuhn
 * tetrahedra, equal-order P1-P1 velocity/pressure with pressure stabilisation
 * C = sum_T tau_T (grad p, grad q)_T, tau_T = beta h^2 / mu_T.  The saddle system is
 *     [ A  B^T ] [u]   [f]
 *     [ B  -C  ] [p] = [g]           (Sec. 5, first display)
 * where A comes from one of three bilinear forms:
 *     SDX_FORM_DECOUPLED  a_tr  = a_sym - (mu div u, div v)    (Sec. 2, eq. newbil)
 *     SDX_FORM_STRAIN     a_sym = (2 mu sym grad u, sym grad v) (Sec. 1, eq. standard)
 *     SDX_FORM_GRADIENT   (mu grad u, grad v)                   (Sec. 4, inconsistent control)
 * The decoupled form is applied as in Sec. 2.2, eq. (equivalence-stencil): a mu-weighted
 * 7-point Laplacian per velocity component on every row, plus the strain cross-couplings
 * only on rows of nodes that touch two viscosities or a traction face.
 *
 * Vectors ("SoA vectors") are four contiguous components u_x, u_y, u_z, p of (n+1)^3
 * doubles each, node (i,j,k) at index i + (n+1)*(j + (n+1)*k).  Velocity components fixed by
 * the boundary conditions ("constrained") must be zero on input and are written as zero.
 * Unless stated otherwise, vector pointers are DEVICE pointers owned by the caller, and every
 * call is asynchronous on the given CUDA stream (NULL = legacy default stream); the library
 * allocates its own work buffers in sdx_create and frees them in sdx_destroy.  Calls on one
 * handle may use its work buffers: order them on one stream (or order the streams), do not
 * run them concurrently.
 *
 * Every function returns SDX_OK (0) or a negative error code; sdx_last_error() gives a
 * message for the calling thread's last failure.  No C++ exception crosses this interface.
 * Errors common to the entry points below, checked before anything is launched: SDX_EINVAL
 * for a NULL handle or vector, a level outside 0..levels-1, or (for the smoothers, cycles and
 * solves) a hierarchy owned by a batch; SDX_ECUDA when a CUDA runtime call fails.  The
 * library cannot see the extent of a vector pointer: a vector shorter than its level's
 * 4*(n+1)^3 entries (3*(n+1)^3 for nodal forcing) is undefined behaviour.
 */
#ifndef SDX_H
#define SDX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define SDX_OK 0
#define SDX_EINVAL (-1)     /* invalid argument (sizes, null pointers, viscosities, ...) */
#define SDX_ENOMEM (-2)     /* a device or host allocation failed; nothing leaked */
#define SDX_ENONFINITE (-3) /* a NaN or Inf appeared in a residual norm */
#define SDX_ENOCONV (-4)    /* maxit reached without meeting rtol; x holds the last iterate */
#define SDX_ECUDA (-5)      /* a CUDA runtime call failed */
#define SDX_ESINGULAR (-6)  /* the coarsest-grid matrix could not be factorised */
#define SDX_ETIMEOUT (-7)   /* a bounded device-side wait gave up (the kernel returned early) */

/* Boundary face types (Sec. 1, eq. boundary).  Faces are ordered -x, +x, -y, +y, -z, +z. */
#define SDX_FACE_DIRICHLET 0 /* u = 0 */
#define SDX_FACE_FREESLIP 1  /* u.n = 0, zero tangential traction */
#define SDX_FACE_TRACTION 2  /* sigma(u,p) n = 0 (natural) */

/* Bilinear forms for the velocity block. */
#define SDX_FORM_DECOUPLED 0
#define SDX_FORM_STRAIN 1
#define SDX_FORM_GRADIENT 2

/* Arithmetic of the multigrid cycle.  The outer residual, the solution update and the
 * coarsest-grid solve are always FP64. */
#define SDX_PREC_FP64 0
#define SDX_PREC_FP32_REFINED 1

/* Outer iteration of sdx_solve. */
#define SDX_OUTER_VCYCLE 0 /* repeated V-cycles (Sec. 5) */
#define SDX_OUTER_FGMRES 1 /* flexible GMRES(restart) right-preconditioned by one V-cycle */

typedef struct sdx_hier* sdx_hier_t; /* opaque, library-owned hierarchy */

typedef struct {
    int n;                  /* cells per side on the finest grid; n = n_coarse * 2^k, k >= 0,
                               n <= 1024 */
    int n_coarse;           /* cells per side on the coarsest grid (>= 2); with coarsening = 0
                               every viscosity interface must lie on a plane of that grid */
    const uint8_t* cell_id; /* HOST array of n^3 subdomain ids, cell (i,j,k) at
                               i + n*(j + n*k); ids must be < n_mu (and < 255) */
    const double* mu;       /* HOST viscosity table indexed by id, all finite and > 0 */
    int n_mu;               /* entries in mu, 1..255 */
    int face[6];            /* SDX_FACE_* for -x, +x, -y, +y, -z, +z */
    int form;               /* SDX_FORM_* on the finest level */
    int coarse_form;        /* SDX_FORM_* on the coarser levels, or -1 for "same as form".
                               (Sec. 5 swaps a_tr for a_sym on the coarse grid.) */
    int prec;               /* SDX_PREC_* for sdx_vcycle and sdx_solve */
    double pspg_beta;       /* stabilisation constant beta (> 0) of tau_T = beta h^2 / mu_T;
                               the paper does not print it; 1/24 (the binding's default) gives
                               the depth-independent multigrid rates of its Sec. 5 table */
    int coarsest_form;      /* SDX_FORM_* on the coarsest level only, or -1 for "same as
                               coarse_form" (with a single level the finest form applies) */
    int coarse_correction;  /* 1: the coarse-grid variant of Sec. 5 - the coarsest solve takes
                               the momentum right-hand side r1 + B^T D r2 (D = diag(mu_b / m_b),
                               m_b the lumped mass, mu_b its mu-weighted mean) so that its a_sym
                               system approximates the a_tr one (A_tr ~ A_sym - B^T D B); needs
                               at least two levels and coarsest_form = SDX_FORM_STRAIN.  The
                               correction is folded into the coarsest inverse when the hierarchy
                               is built, so a cycle costs the same.  0: no correction. */
    int coarsening;         /* how coarse cells get their viscosity id from their 8 children:
                               0 = every viscosity interface must lie on a plane of the coarsest
                               grid (the 8 children agree; SDX_EINVAL otherwise); 1 = interfaces
                               the coarse grids do not resolve (a level set cutting the cells,
                               Sec. 2.2 closing remark): the id whose viscosity most children
                               have, a tie going to the larger viscosity (the smallest such id).
                               The finest operator is exact either way; the coarse levels only
                               precondition. */
} sdx_desc;

typedef struct {
    int iterations; /* V-cycles applied (each FGMRES iteration applies one) */
    int restarts;   /* FGMRES restarts (0 for SDX_OUTER_VCYCLE) */
    double res0;    /* ||b - K x0||_2 over free DoFs */
    double res;     /* final ||b - K x||_2 */
    double bnorm;   /* ||b||_2 */
    int status;     /* same value as the call's return code */
} sdx_stats;

/* Build the grid hierarchy n, n/2, ..., n_coarse: cell viscosities, boundary masks,
 * interface-row lists, device work buffers (library-owned) and the dense FP64 inverse of the
 * coarsest-grid saddle matrix (bordered by the pressure-mean row int q/mu = 0 when no face is
 * a traction face).  Synchronous.  Paper: Sec. 4.2.3 (mesh), Sec. 5 (direct coarse solve).
 * The coarsest grid may have at most 12000 unknowns (n_coarse <= 13 or so), since its saddle
 * matrix is inverted densely.
 * Errors: SDX_EINVAL for bad sizes/ids/viscosities, interfaces not resolved on the coarsest
 * grid or a coarsest grid too large, SDX_ENOMEM, SDX_ESINGULAR, SDX_ECUDA.  On error *out is set to NULL. */
int sdx_create(const sdx_desc* desc, sdx_hier_t* out);

/* Release every buffer of the hierarchy.  Synchronises the device first.  NULL is a no-op.
 * A hierarchy obtained from sdx_batch_instance is refused with SDX_EINVAL (the batch owns it). */
int sdx_destroy(sdx_hier_t h);

/* Number of levels, and nodes / free DoFs of one level (0 = finest). */
int sdx_levels(sdx_hier_t h, int* levels);
int sdx_level_size(sdx_hier_t h, int level, int* n, int64_t* nodes, int64_t* free_dofs);

/* Host query: mask[4*(n+1)^3] set to 1 at constrained DoFs of the level, 0 elsewhere. */
int sdx_constraint_mask(sdx_hier_t h, int level, uint8_t* mask_host);

/* Host query: iface[(n+1)^3] set to 1 at interface rows (nodes that get the strain
 * cross-couplings in the decoupled form, Sec. 2.2), 0 elsewhere. */
int sdx_interface_mask(sdx_hier_t h, int level, uint8_t* iface_host);

/* y = K x on one level (device SoA vectors of that level's size), with the level's form.
 * Paper: Sec. 2.2 eq. (equivalence-stencil) for the decoupled form; Sec. 5 saddle matrix. */
int sdx_apply(sdx_hier_t h, int level, const double* x, double* y, void* stream);

/* r = b - K x on one level. */
int sdx_residual(sdx_hier_t h, int level, const double* b, const double* x, double* r,
                 void* stream);

/* Right-hand side of the finest level from nodal forcing f (device, three components of
 * (n+1)^3): velocity rows m_b f(x_b) with the lumped mass m_b = int lambda_b; pressure rows
 * the stabilisation term g_b = -sum_T tau_T int_T f_h . grad lambda_b (f_h: P1 interpolant).
 * Constrained rows are zero. */
int sdx_rhs(sdx_hier_t h, const double* f_nodal, double* b, void* stream);

/* One Uzawa smoothing step (Sec. 5, eq. Uzawa_smooth) on one level, in place on x:
 * symmetric red-black Gauss-Seidel on A (colours red, black, red; couplings between
 * velocity components of same-coloured nodes taken from the values before the colour pass),
 * then forward red-black Gauss-Seidel on C p = B u - g with relaxation 0.3.  FP64. */
int sdx_uzawa(sdx_hier_t h, int level, const double* b, double* x, void* stream);

/* One colour pass of the Uzawa smoother on one level, in place on x (FP64): which = 0 is
 * the velocity Gauss-Seidel pass on A u = f - B^T p over nodes of the given colour
 * (0: i+j+k even, 1: odd), which = 1 the relaxed pressure pass on C p = B u - g.  sdx_uzawa
 * is velocity passes 0, 1, 0 followed by pressure passes 0, 1.  Paper: Sec. 5. */
int sdx_smooth_pass(sdx_hier_t h, int level, int which, int colour, const double* b, double* x,
                    void* stream);

/* FP32 versions of sdx_apply and sdx_smooth_pass on FP32 SoA vectors (float, same layout):
 * the arithmetic of the FP32 multigrid cycle used by SDX_PREC_FP32_REFINED.  They need a
 * hierarchy created with prec = SDX_PREC_FP32_REFINED (SDX_EINVAL otherwise). */
int sdx_apply_f32(sdx_hier_t h, int level, const float* x, float* y, void* stream);
int sdx_smooth_pass_f32(sdx_hier_t h, int level, int which, int colour, const float* b, float* x,
                        void* stream);

/* `steps` FP32 Uzawa smoothing steps (as sdx_uzawa, 1 <= steps <= 1000) on one level, in place
 * on the FP32 vector x, with exactly the launches the FP32 V-cycle uses on that level: one
 * launch per pass, or, on levels of at most SDX_CLUSTER_MAX_NODES nodes (environment variable
 * read when the hierarchy is created; default 0 = never), all steps in one thread-block
 * cluster with hardware cluster barriers between the colour passes.  Needs a hierarchy created
 * with prec = SDX_PREC_FP32_REFINED.  Paper: Sec. 5, eq. (Uzawa_smooth). */
int sdx_uzawa_f32(sdx_hier_t h, int level, const float* b, float* x, int steps, void* stream);

/* Allocation-free variant of the velocity pass of sdx_smooth_pass (which = 0), FP64.
 * The paper has no counterpart; this exists for callers that cannot allocate device memory at
 * the point of the call - for example code running in a phase where cudaMalloc is forbidden
 * because it would synchronise the device or because device memory is budgeted up front - and
 * that do not want the pass to depend on a scratch buffer sized by the hierarchy.  It computes
 * exactly what sdx_smooth_pass(h, level, 0, colour, b, x, stream) computes, but the new
 * values of the boundary/interface rows are staged in a fixed array compiled into the
 * library (SDX_NOALLOC_MAX_ROWS rows, 3 doubles each: 1.5 MiB that every GPU which loads the
 * library holds until the process exits).  The call allocates nothing.
 *   - Decoupled and gradient forms only: the strain form's pass needs a full-grid scratch
 *     vector and is rejected with SDX_EINVAL.
 *   - A level whose colour has more than SDX_NOALLOC_MAX_ROWS boundary/interface rows is
 *     rejected with SDX_EINVAL before anything is launched (see sdx_last_error()).
 *   - The first call on a device looks up the array's device address (once per device, with
 *     that device current); make that first call before any stream capture.  The address is
 *     kept for the life of the process: after cudaDeviceReset (or anything else that destroys
 *     and recreates the device's primary context) the kept address is stale, so do not call
 *     this entry point again in that process.
 *   - All calls share the one array.  Nothing in it needs to start at zero (each call writes
 *     every entry it later reads), but calls whose executions overlap on the GPU (different
 *     streams, different hierarchies) race on it: serialise them. */
#define SDX_NOALLOC_MAX_ROWS 65536
int sdx_smooth_pass_noalloc(sdx_hier_t h, int level, int colour, const double* b, double* x,
                            void* stream);

/* Transfers between level l (fine) and l+1 (coarse), standard nested P1 operators:
 * sdx_restrict writes b_coarse = P^T r_fine; sdx_prolong_add does x_fine += P e_coarse.
 * Constrained DoFs are masked on both levels.  FP64. */
int sdx_restrict(sdx_hier_t h, int level, const double* r_fine, double* b_coarse, void* stream);
int sdx_prolong_add(sdx_hier_t h, int level, const double* e_coarse, double* x_fine,
                    void* stream);

/* One variable V-cycle (V_var(3,3): 3 + 2k pre- and post-smoothing steps k levels below the
 * finest) on the finest level, in place on x, in the hierarchy's precision.  FP32 mode runs
 * the cycle on r = b - K x in FP32 and adds the correction in FP64.  Paper: Sec. 5. */
int sdx_vcycle(sdx_hier_t h, const double* b, double* x, void* stream);

/* Solve K x = b to ||b - K x||_2 <= rtol ||b||_2 (free DoFs), starting from the x passed in.
 * outer: SDX_OUTER_VCYCLE or SDX_OUTER_FGMRES (restart = Krylov basis size, >= 1; ignored
 * for V-cycles).  Synchronises the stream once per iteration to test convergence.  stats may
 * be NULL.  Returns SDX_ENOCONV if maxit iterations did not meet rtol, SDX_ENONFINITE if a
 * residual norm was NaN/Inf (x is then the last finite iterate or garbage, stats filled),
 * SDX_ETIMEOUT if a fused smoothing launch gave up a grid barrier after its bounded wait
 * (reported at the next synchronisation; x is then not meaningful).  With b = 0 the target
 * is 0: from x = 0 the call returns at once (0 iterations); from any other x it iterates,
 * driving x towards 0, until maxit (SDX_ENOCONV) - pass x = 0 for a zero right-hand side.
 * The smoothing steps of small levels may run fused in one launch when the environment sets a
 * node limit at hierarchy creation (SDX_CLUSTER_MAX_NODES / SDX_CLUSTER_MAX_NODES_FP64: one
 * thread-block cluster; SDX_COOP_MAX_NODES: a cooperative grid launch; SDX_NO_COOP=1 disables
 * both); by default every level uses one launch per pass.  Every variant gives the same bits. */
int sdx_solve(sdx_hier_t h, const double* b, double* x, double rtol, int maxit, int outer,
              int restart, sdx_stats* stats, void* stream);

/* As sdx_solve, but b_host and x_host are HOST arrays (pinned or pageable): copies b and x
 * to library buffers, solves, copies x back, and synchronises the stream before returning. */
int sdx_solve_host(sdx_hier_t h, const double* b_host, double* x_host, double rtol, int maxit,
                   int outer, int restart, sdx_stats* stats, void* stream);

/* ------------------------------------------------------------------ batched solves
 * A batch holds `count` independent problems (grid sizes, viscosity layouts and boundary
 * faces may differ; form, coarse_form and prec must be the same) and advances them
 * together: every phase of the V-cycle (a colour pass, the special rows of a colour, a
 * residual, a transfer, the coarsest-grid solves) is one persistent launch over the work of
 * all instances, the whole V-cycle is one CUDA graph, and the outer iteration is flexible
 * GMRES per instance with all Krylov steps in lock step (converged instances drop out of
 * every launch).  The arithmetic per instance is the one of sdx_vcycle / sdx_solve.
 * Paper: Sec. 5 (V_var(3,3) Uzawa multigrid, direct coarse solve) applied to many problems;
 * the batching itself has no counterpart in the paper. */
typedef struct sdx_batch* sdx_batch_t; /* opaque, library-owned */

/* Build the hierarchies of descs[0..count-1] (1 <= count <= 256) and the batch's own
 * concatenated work vectors.  autotune != 0 times candidate block shapes (64..512 threads per
 * block, persistent grids of one or two waves of resident blocks) of the colour-pass and
 * residual launches on every level and keeps the fastest.  Synchronous.  Errors as sdx_create, plus SDX_EINVAL
 * when the descriptors disagree on form, coarse_form, coarsest_form, coarse_correction or prec.  On error *out is NULL. */
int sdx_batch_create(const sdx_desc* descs, int count, int autotune, sdx_batch_t* out);

/* Release the batch and every hierarchy in it (synchronises the device).  NULL is a no-op. */
int sdx_batch_destroy(sdx_batch_t b);

/* Finest-level size of one instance, as sdx_level_size(level 0). */
int sdx_batch_size(sdx_batch_t b, int instance, int* n, int64_t* nodes, int64_t* free_dofs);

/* Hierarchy of one instance, owned by the batch (valid until sdx_batch_destroy; never pass it
 * to sdx_destroy).  It serves the queries, sdx_rhs, sdx_apply, sdx_residual, the transfers
 * and the sdx_guess_* calls; calls that need the hierarchy's own work vectors (smoothers,
 * V-cycles, solves) return SDX_EINVAL on it, since the batch keeps its own. */
int sdx_batch_instance(sdx_batch_t b, int instance, sdx_hier_t* out);

/* Block shape chosen for one batch level: threads per block and blocks of the colour-pass
 * launches and of the residual launches (any output pointer may be NULL). */
int sdx_batch_shape(sdx_batch_t b, int level, int* tpb_pass, int* grid_pass, int* tpb_residual,
                    int* grid_residual);

/* One V-cycle of every instance, in place: x[i] += M_i (b[i] - K_i x[i]), the same
 * arithmetic as sdx_vcycle on each instance's own hierarchy.  b and x are HOST arrays of
 * `count` DEVICE pointers to SoA vectors of each instance's finest level. */
int sdx_batch_vcycle(sdx_batch_t b, const double* const* bvec, double* const* x, void* stream);

/* Solve every instance to ||b_i - K_i x_i|| <= rtol ||b_i|| with FGMRES(restart)
 * right-preconditioned by one V-cycle, starting from the x[i] passed in.  stats (may be
 * NULL) receives `count` entries.  Synchronises the stream once per Krylov step.  Returns
 * SDX_OK when every instance converged, SDX_ENOCONV if some hit maxit, SDX_ENONFINITE if a
 * residual became NaN/Inf (per-instance status in stats).  b and x as in sdx_batch_vcycle. */
int sdx_batch_solve(sdx_batch_t b, const double* const* bvec, double* const* x, double rtol,
                    int maxit, int restart, sdx_stats* stats, void* stream);

/* ------------------------------------------------------------------ learned initial guess
 * A small 3D U-Net predicts an initial iterate from the viscosity layout and the forcing; the
 * solver then runs to the same residual as from zero.  The paper has no counterpart.
 * The network works on the n^3 cells (n a multiple of 4): tensors are [n^3][C] (cell
 * i + n*(j + n*k), C channels contiguous), BF16 activations, FP32 accumulation.  Layers
 * (3x3x3 convolutions, zero padding, weights [27][C_out][C_in], tap t = (dz+1)*9 + (dy+1)*3 +
 * (dx+1) reading the input at offset (dx, dy, dz)):
 *   a1 = relu(conv(x, 16->16)), a2 = relu(conv(a1, 16->16)),
 *   a3 = relu(conv(pool(a2), 16->32)), a4 = relu(conv(a3, 32->32)),
 *   a5 = relu(conv(pool(a4), 32->64)),
 *   a6 = relu(conv(up(a5), 64->32) + a4), a7 = relu(conv(a6, 32->32)),
 *   a8 = relu(conv(up(a7), 32->16) + a2), a9 = relu(conv(a8, 16->16)),
 *   y  = conv(a9, 16->16)  (channels 0..3: u_x, u_y, u_z, p over the forcing scale)
 * pool = mean of 2x2x2 cells, up = nearest neighbour; every convolution adds a bias.
 * Parameters (221456 FP32 values) are stored layer by layer, W then b.  Input channels:
 * log10 mu, the cell mean of the nodal forcing / fscale (3), 1, zeros (fscale = max |f|).
 * Loss: sum over cells and channels 0..3 of (y - target)^2 / (4 n^3); optimiser: Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) on the mean gradient of each mini-batch.  Convolutions
 * and weight gradients run on the tensor cores (tcgen05, BF16 in, FP32 accumulate). */
typedef struct sdx_net* sdx_net_t; /* opaque, library-owned network with its optimiser state */

/* Parameter count of the network (221456). */
int64_t sdx_net_param_count(void);

/* Create a network with He-normal weights drawn from `seed` and zero biases.  Synchronous. */
int sdx_net_create(uint64_t seed, sdx_net_t* out);
int sdx_net_destroy(sdx_net_t net);

/* Copy the FP32 parameters to / from a HOST array of sdx_net_param_count() floats;
 * sdx_net_set_params also resets the optimiser state.  Synchronous. */
int sdx_net_get_params(sdx_net_t net, float* params_host);
int sdx_net_set_params(sdx_net_t net, const float* params_host);

/* y[n^3][16] (FP32, device) = network(x[n^3][16] (BF16 bit patterns, device)).  Synchronises
 * the stream; SDX_ETIMEOUT if a tensor-core wait gave up. */
int sdx_net_forward(sdx_net_t net, int n, const uint16_t* x, float* y, void* stream);

/* Loss and gradient of one sample (x as above, target [n^3][16] FP32, device): *loss_host and
 * grads_host (sdx_net_param_count() floats, may be NULL).  Synchronises the stream. */
int sdx_net_loss_grad(sdx_net_t net, int n, const uint16_t* x, const float* target,
                      double* loss_host, float* grads_host, void* stream);

/* Train on `count` samples stored back to back (x: count x n^3 x 16 BF16, target: count x
 * n^3 x 16 FP32, device) for `epochs` passes in seeded random order, Adam steps on
 * mini-batches of `batch` samples with learning rate lr; loss_history_host (may be NULL)
 * receives the mean loss of every epoch.  Synchronises once per epoch. */
int sdx_net_train(sdx_net_t net, int n, int count, const uint16_t* x, const float* target,
                  int epochs, int batch, float lr, uint64_t seed, double* loss_history_host,
                  void* stream);

/* The tensor-core convolution itself (for testing): y[n^3][cout] (FP32) = conv(x[n^3][cin],
 * w[27][cout][cin]) + bias (may be NULL), ReLU if relu != 0; x and w BF16 bit patterns.
 * Shapes (cin, cout) in {(16,16), (16,32), (32,16), (32,32), (32,64), (64,32)}.
 * sdx_conv3_wgrad adds dw[t][co][ci] += sum_v dz[v][co] x[v + off_t][ci] (dz BF16 [n^3][cout],
 * dw FP32).  Both synchronise the stream. */
int sdx_conv3(int n, int cin, int cout, const uint16_t* x, const uint16_t* w, const float* bias,
              int relu, float* y, void* stream);
int sdx_conv3_wgrad(int n, int cin, int cout, const uint16_t* x, const uint16_t* dz, float* dw,
                    void* stream);
/* Input gradient of the convolution, as the network's backward pass computes it (for testing):
 * dx[v][ci] (FP32) = sum over taps t and output channels co of W[t][co][ci] dz[v - off_t][co],
 * i.e. the forward kernel run on the weights flipped in the taps and transposed in the channels
 * (converted to BF16 on the device).  dz: BF16 [n^3][cout]; w: FP32 [27][cout][cin] (the layout
 * of the network's parameters); same shapes as sdx_conv3.  Allocates its flipped-weight
 * buffer and synchronises the stream.  Paper: no counterpart (the learned initial guess is an
 * addition to the method). */
int sdx_conv3_dgrad(int n, int cin, int cout, const uint16_t* dz, const float* w, float* dx, void* stream);

/* Network input of a hierarchy's finest grid (n a multiple of 4) from the nodal forcing f
 * (device, 3 x (n+1)^3): x[n^3][16] (device, BF16) and *fscale_host = max |f| (1 if f = 0).
 * Synchronises the stream. */
int sdx_guess_features(sdx_hier_t h, const double* f_nodal, uint16_t* x, double* fscale_host,
                       void* stream);

/* Training target from a solution (device SoA vector of the finest level): t[n^3][16] (FP32)
 * with the cell means of 100 u_x, 100 u_y, 100 u_z and p - (mean of p over the nodes), all
 * over fscale, in channels 0..3, zeros elsewhere (the factor 100 brings the velocities of the
 * blob-forced problems to the size of the pressures).  Synchronises the stream. */
int sdx_guess_target(sdx_hier_t h, const double* x_solution, double fscale, float* target,
                     void* stream);

/* Initial guess x0 (device SoA vector of the finest level) for the forcing f: features,
 * network, then every node takes the mean of the prediction over its cells, times fscale;
 * constrained components are zero.  Asynchronous; the network's scratch is sized for the
 * last grid it saw (resizing synchronises the device). */
int sdx_guess_predict(sdx_hier_t h, sdx_net_t net, const double* f_nodal, double* x0,
                      void* stream);

/* Make a predicted iterate safe to start from: `steps` FP64 Uzawa smoothing steps on the
 * finest level (as sdx_uzawa) with right-hand side b, then x is replaced by its
 * residual-minimising multiple alpha x, alpha = (Kx, b) / (Kx, Kx), so that
 * ||b - K x|| <= ||b|| always holds.  Asynchronous.  Not for batch-owned hierarchies. */
int sdx_guess_refine(sdx_hier_t h, const double* b, double* x, int steps, void* stream);

/* ------------------------------------------------------------------ P1-P0 scheme
 * The stabilised lowest-order pair of Sec. 3.1-3.2: P1 velocity (the same velocity block,
 * forms, boundary conditions and hierarchy rules as above) and one pressure per tetrahedron,
 * with the interior-penalty stabilisation of eq. (stabc),
 *     c(p, q) = gamma sum_i 1/(2 mu_i) sum over the interior facets F of subdomain i of
 *               |T1||T2| / (|T1| + |T2|) [p]_F [q]_F
 * (no penalty across the viscosity interface or on the domain boundary; the paper uses
 * gamma = 1, Sec. 4.2), and b(v, q) = -(div v, q).  Vectors are 3 (n+1)^3 velocity values
 * (u_x, u_y, u_z as above) followed by 6 n^3 pressures, tetrahedron s of cell (i, j, k) at
 * s * n^3 + i + n (j + n k), s the axis permutation of the Kuhn path c, c + e_s1, c + e_s1 + e_s2,
 * c + (1,1,1) in the order (0,1,2), (0,2,1), (1,0,2), (1,2,0), (2,0,1), (2,1,0).  FP64 only.
 * Solver: the V_var(3,3) Uzawa cycle with the red-black velocity smoother above and a relaxed
 * Jacobi pressure step on the 1/mu-weighted P0 mass (p += 0.6 (mu_T / |T|) (B u - C p - g)_T),
 * P0 pressures transferred by embedding a coarse tetrahedron into its eight children; FGMRES or
 * plain cycles outside; direct coarsest solve (at most 12000 unknowns). */
typedef struct sdx_p0* sdx_p0_t; /* opaque, library-owned */

/* Build the hierarchy (desc->prec must be SDX_PREC_FP64; pspg_beta is not used and
 * coarse_correction must be 0) with penalty constant gamma > 0.  Synchronous.  Errors as
 * sdx_create, plus SDX_EINVAL for gamma <= 0 or not finite.  The handle owns every work buffer
 * (the per-level vectors, the coarsest inverse, the Krylov basis allocated on the first
 * FGMRES solve) until sdx_p0_destroy, which synchronises the device; NULL is a no-op.
 * The calls below follow the conventions at the top of this file: device vectors owned by the
 * caller, asynchronous on the stream unless stated, SDX_EINVAL for a NULL handle or vector or a
 * level out of range, SDX_ECUDA when a launch fails. */
int sdx_p0_create(const sdx_desc* desc, double gamma, sdx_p0_t* out);
int sdx_p0_destroy(sdx_p0_t h);
/* Cells per side, nodes, tetrahedra and free unknowns of one level. */
int sdx_p0_size(sdx_p0_t h, int level, int* n, int64_t* nodes, int64_t* tets, int64_t* free_dofs);
/* y = K x and r = b - K x on one level (device vectors of 3 (n+1)^3 + 6 n^3 doubles). */
int sdx_p0_apply(sdx_p0_t h, int level, const double* x, double* y, void* stream);
int sdx_p0_residual(sdx_p0_t h, int level, const double* b, const double* x, double* r, void* stream);
/* Finest-level right-hand side: velocity rows as sdx_rhs (lumped mass times the nodal
 * forcing), pressure rows zero (the interior-penalty form has no consistent load). */
int sdx_p0_rhs(sdx_p0_t h, const double* f_nodal, double* b, void* stream);
/* One Uzawa smoothing step on one level, in place on x. */
int sdx_p0_uzawa(sdx_p0_t h, int level, const double* b, double* x, void* stream);
/* One V-cycle on the finest level: x += M (b - K x). */
int sdx_p0_vcycle(sdx_p0_t h, const double* b, double* x, void* stream);
/* Solve as sdx_solve (same arguments and return codes; synchronises the stream, since the
 * convergence test and FGMRES's small least-squares problem run on the host). */
int sdx_p0_solve(sdx_p0_t h, const double* b, double* x, double rtol, int maxit, int outer, int restart,
                 sdx_stats* stats, void* stream);
/* Local flux post-process (Sec. 3.2, remark after eq. stabc) of a finest-level vector x:
 * flux[4 t + m] = int over the facet of tetrahedron t opposite its path vertex m of
 * u_h . n_T + Delta j, Delta j integrated = gamma / (2 mu) |T||T_F| / (|T| + |T_F|) (p_T - p_F)
 * on facets inside one viscosity (outward from t), and balance[t] = the sum of t's four
 * fluxes, zero for a solution of the discrete problem (element-wise mass conservation).
 * flux: 4 * 6 n^3 doubles, balance: 6 n^3 doubles (device). */
int sdx_p0_fluxes(sdx_p0_t h, const double* x, double* flux, double* balance, void* stream);

/* Number of CUDA kernels this library has launched in the process so far (all
 * hierarchies, all threads); used to count the kernels of a timed region. */
int64_t sdx_kernel_launches(void);

/* Message describing the calling thread's last error (never NULL). */
const char* sdx_last_error(void);

/* Static description of an error code (never NULL). */
const char* sdx_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SDX_H */
