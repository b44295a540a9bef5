/*
 * helm.h -- C-ABI of libhelm: multi-source frequency-domain Helmholtz solves
 * on one GB300 (sm_103a) with a shifted-Laplacian multigrid preconditioned
 * block flexible GMRES.
 *
 * Problem (Treister & Haber, Sec. 2.1 Eq. helm and Sec. 2.4 Eq.
 * LinearSystem), in this library's sign convention:
 *
 *     A u := -Lap_h u - omega^2 m (1 - i gamma) u = q,
 *
 * with the second-order 5-point (2D) / 7-point (3D) Laplacian on the nodes
 * of a regular grid, Dirichlet zero beyond the node grid, squared slowness m
 * and a dimensionless attenuation gamma that carries the absorbing layer.
 * (The paper writes Lap_h u + omega^2 (1 - i gamma_p/omega) m u = q; so
 * gamma = gamma_p/omega and u = -u_paper.)
 *
 * Preconditioner (Sec. 4): one multigrid V-cycle for the shifted operator
 * M = A with gamma -> gamma + shift, Galerkin coarse operators
 * M_{l+1} = P^T M_l P with bi/trilinear P, damped Jacobi relaxation and a
 * dense LU (stored as the inverse) on the coarsest grid (Sec. 4, Alg.
 * "Two-grid cycle"; Sec. 5.3 settings: 2 pre + 2 post sweeps, weight 0.8).
 * Krylov method: block FGMRES(m) (Sec. 5.3), run on groups of `block`
 * right-hand sides that advance in lock step and share every kernel launch.
 *
 * Layouts
 *   Node index: x1 fastest, then x2, then x3; n[k] cells give n[k]+1 nodes.
 *   ABI block (helm_solve, helm_adjoint): complex128 (interleaved re, im),
 *     N x s column-major, i.e. column j (one right-hand side) is the N
 *     contiguous complex values Q[j*N .. j*N+N-1].
 *   Internal block (component entry points below): node-major with the
 *     right-hand sides innermost, x[node*s + j]; complex128 or complex64 as
 *     the `prec` argument says.
 *
 * Ownership and ordering
 *   The caller owns every buffer it passes; the context owns its hierarchy
 *   and workspace (device memory allocated with cudaMalloc at set-up and,
 *   when a larger s is first seen, at the first solve with that s).  All
 *   device work is enqueued on the stream given to helm_setup; every call
 *   returns after that stream has been synchronised.  Pointers marked
 *   "device" must be device (or managed) memory of the current device.
 *
 * Errors
 *   Every call returns a helm_status; no exception crosses the ABI.  On any
 *   status other than HELM_OK, helm_last_error() describes it.  A solve that
 *   stops early (HELM_NOT_CONVERGED, HELM_ERR_NONFINITE) still writes the
 *   best iterate to U and fills `info`.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_ctx helm_ctx;

typedef enum {
    HELM_OK = 0,
    HELM_ERR_ARG = 1,          /* bad argument (sizes, pointers, levels)      */
    HELM_ERR_NOMEM = 2,        /* device or host allocation failed            */
    HELM_ERR_CUDA = 3,         /* a CUDA runtime call failed                  */
    HELM_NOT_CONVERGED = 4,    /* iteration cap reached; U = best iterate     */
    HELM_ERR_NONFINITE = 5,    /* NaN/Inf met in an FP64 residual norm        */
    HELM_ERR_BREAKDOWN = 6     /* singular coarsest operator or Krylov block  */
} helm_status;

typedef enum {
    HELM_PLAIN_C128 = 0,        /* every step in complex128 (FP64)             */
    HELM_MIXED_C64 = 1,         /* V-cycle in complex64 with FP32 accumulation;
                                   A*Z, residuals, orthogonalisation, QR and
                                   least squares in FP64                       */
    HELM_MIXED_C64_LEARNED = 2  /* HELM_MIXED_C64 plus the learned stage       */
} helm_prec;

typedef struct {
    int dim;                 /* 2 or 3                                          */
    int n[3];                /* cells per axis (x1, x2, x3); nodes = n[k]+1;
                                every n[k] divisible by 2^(levels-1)            */
    double h;                /* grid spacing (same on every axis)               */
    double omega;            /* angular frequency                               */
    double shift;            /* beta added to gamma in the preconditioner (0.5) */
    int levels;              /* multigrid levels, >= 1 (1 = dense solve only)   */
    int pre, post;           /* Jacobi sweeps before / after the coarse
                                correction (2, 2)                               */
    double jacobi_w;         /* Jacobi damping (0.8)                            */
    int restart;             /* FGMRES(m): block steps per restart cycle (10)   */
    int block;               /* right-hand sides per Krylov block (>= 1)        */
    int max_restarts;        /* restart cycles before HELM_NOT_CONVERGED        */
    helm_prec prec;          /* precision policy                                */
    const void* learned_weights; /* device blob of the learned stage (layout:
                                    helm_learned_layer below), caller-owned,
                                    must outlive the context; required by
                                    HELM_MIXED_C64_LEARNED (2D only)            */
    int coarse_tf32x3;       /* complex64 coarsest solve on the tensor cores:
                                0 = one FP16 product (11 significant bits,
                                power-of-two scales of the inverse and of
                                each right-hand side; ~1e-3 relative) on the
                                5th-generation tensor cores (tcgen05.mma,
                                TMA-fed shared memory, accumulator in tensor
                                memory);
                                1 = three tf32 products on hi/lo splits
                                (FP32-class, mma.sync);
                                2 = the FP16 product of 0 on mma.sync tiles
                                (the earlier kernel, kept for comparison)    */
    int cycle_gamma;         /* 1 = V-cycle, 2 = W-cycle (two coarse visits per
                                level, Sec. 4), 3 = K-cycle (Sec. 5.3: each
                                coarse system solved by two flexible Krylov
                                steps preconditioned by the next cycle; here
                                per column, GCR(2); FGMRES only; s <= 256)     */
    int krylov;              /* 0 = block FGMRES(restart); 1 = block BiCGSTAB
                                (Sec. 5.3 "W-BiCG", El Guennouni et al.; needs
                                a fixed preconditioner: not with the learned
                                stage, and with the complex64 cycle only for
                                block <= 2 -- measured: larger blocks diverge
                                under the cycle's FP32 rounding, while the
                                complex128 cycle converges at any block);
                                iterations capped at restart * max_restarts
                                per run, max_restarts + 1 runs                  */
    int graphs;              /* block FGMRES without the learned stage: replay
                                each Krylov step's device work (cycle, A Z_j,
                                Gram-Schmidt, first QR Gram and their copies
                                to the host) from a CUDA graph captured on the
                                step's first use. 0 = launch directly,
                                1 = always, 2 = when N * s <= 4,194,304
                                (launch-bound sizes).  Never while the
                                profiler is on (it times single launches).
                                Results are identical either way.            */
    int orth;                /* block FGMRES orthogonalisation of each new
                                block W = A Z_j against the basis and its own
                                QR (Sec. 5.3 block FGMRES; the paper leaves
                                the scheme open):
                                0 = one classical Gram-Schmidt pass and one
                                Cholesky QR pass, each repeated only when its
                                rounding could leave the new basis block less
                                orthogonal than 1e-11 (second Gram-Schmidt
                                pass when u / sin(theta_min) * kappa_F(W')
                                > 1e-11, second Cholesky QR pass when
                                u * kappa_F(W')^2 > 1e-11, u = 2^-53 in FP64
                                and 2^-46 for the float-pair arithmetic of
                                the complex64 path);
                                1 = always two passes of each (CGS2 +
                                CholQR2)                                      */
} helm_params;

typedef struct {
    int* iters;     /* per column: preconditioner applications (the paper's
                       #Cyc, Sec. 5.3 table), caller-owned host array of s   */
    double* relres; /* per column: true ||q - A u|| / ||q|| in FP64 (0 for a
                       zero column), caller-owned host array of s             */
    int* status;    /* per column: helm_status, caller-owned host array of s  */
} helm_info;

/* Fill p with the defaults of Sec. 5.3 (levels 3, V(2,2), weight 0.8,
   restart 10) plus shift 0.5, block 8, max_restarts 50, HELM_PLAIN_C128,
   coarse_tf32x3 0, cycle_gamma 1, krylov 0, graphs 2, orth 0. */
void helm_default_params(helm_params* p);

/* Set up the hierarchy for one (m, gamma, omega) (Sec. 4: set-up once, reused
   by every right-hand side and by the adjoint solve).
   m, gamma_tilde: device float64 arrays of N = prod(n[k]+1) node values,
   copied; cuda_stream: a cudaStream_t (NULL = legacy default stream).
   Builds A's and M's fine-level coefficients, the Galerkin coefficients of
   every coarse level, the Jacobi inverse diagonals and the inverse of the
   coarsest operator (Gauss-Jordan with partial pivoting; FP64 for
   HELM_PLAIN_C128, FP32 for the complex64 cycles).
   Returns HELM_ERR_ARG for bad sizes, HELM_ERR_BREAKDOWN when the coarsest
   operator is singular. */
helm_status helm_setup(const double* m, const double* gamma_tilde,
                       const helm_params* p, void* cuda_stream, helm_ctx** out);

/* Solve A U = Q for s right-hand sides to per-column relative residual tol
   (FP64, true residual), X_0 = 0 (Sec. 5.3: block FGMRES preconditioned by
   the shifted-Laplacian cycle).  Q, U: device complex128, ABI layout, N x s.
   A zero column gives a zero solution with relres 0.  info may be NULL.
   s = 0 returns HELM_OK and touches nothing (Q and U may then be NULL);
   s < 0, tol <= 0, or a NULL Q or U with s > 0 gives HELM_ERR_ARG. */
helm_status helm_solve(helm_ctx* ctx, const void* Q, int s, double tol,
                       void* U, helm_info* info);

/* Solve A^H L = B (the adjoint solve of the sensitivity, Sec. 2.4 Eq.
   fwisens; Sec. 4 last paragraph: same hierarchy).  A is complex symmetric,
   so L = conj(A^{-1} conj(B)).  Same layout and semantics as helm_solve. */
helm_status helm_adjoint(helm_ctx* ctx, const void* B, int s, double tol,
                         void* L, helm_info* info);

/* helm_solve with HOST complex128 buffers (ABI layout): copies Q to the
   device, solves, copies U back, all on the context's stream.  Pinned host
   memory makes the copies asynchronous DMA; pageable memory works too.  The
   device staging of Q and U is owned by the context and holds as many
   columns as its workspace; s = 0 and bad arguments behave as in
   helm_solve. */
helm_status helm_solve_host(helm_ctx* ctx, const void* Q_host, int s,
                            double tol, void* U_host, helm_info* info);

/* Solve several independent problems (contexts, possibly different grids,
   frequencies and precisions; the uneven batches of many sources and
   frequencies of Sec. 2.1's misfit): problem k solves ctxs[k] with Q[k]
   (s[k] columns, device, ABI layout) into U[k], infos[k] (infos may be NULL).
   Problems are taken longest first under a cost model (nodes x columns x
   omega h max(n), x4 for the FP64 path) by HELM_BATCH_WORKERS host workers
   (environment variable, default 4); each runs on its context's stream, so
   contexts created with distinct streams overlap on the GPU.  A context must
   appear at most once per batch.  Returns the first non-OK status in problem
   order (every problem is attempted). */
helm_status helm_solve_batch(helm_ctx* const* ctxs, const void* const* Q,
                             const int* s, int nprob, double tol,
                             void* const* U, helm_info* infos);

void helm_destroy(helm_ctx* ctx);

/* Message of the last error of ctx (or of this thread when ctx is NULL). */
const char* helm_last_error(const helm_ctx* ctx);

/* ---------------------------------------------------------------------
 * Component entry points (internal layout, device pointers).  They expose
 * the hot-path steps one by one so that each can be checked on its own.
 * `prec`: 0 = complex128 vectors and FP64 arithmetic, 1 = complex64 vectors
 * and FP32 arithmetic (coefficients rounded from the FP64 set-up).
 * Level 0 is the fine grid; level levels-1 the coarsest.  An output must
 * not share memory with an input of the same call (the stencil kernels read
 * the neighbours of the nodes they write); helm_prolong_add, which updates u
 * in place, is the exception.
 * ------------------------------------------------------------------- */

/* Nodes per axis (nodes[3], unused axes 1) and node count of a level. */
helm_status helm_level_shape(const helm_ctx* ctx, int level, int* nodes,
                             long long* count);

/* y = Op x for s columns.  op = 0: A (level 0 only), op = 1: M_level
   (fine: 5/7-point stencil, Sec. 2.4; coarse: Galerkin P^T M P, Sec. 4). */
helm_status helm_apply(helm_ctx* ctx, int level, int op, int prec,
                       const void* x, void* y, int s);

/* Damped Jacobi on M_level (Sec. 5.3): `sweeps` times
   u <- u + w D^{-1} (f - M u), starting from u_in (NULL = zero). */
helm_status helm_smooth(helm_ctx* ctx, int level, int prec, const void* u_in,
                        const void* f, void* u_out, int s, int sweeps);

/* rc = P^T (f - M_level u) on level+1 (Alg. "Two-grid cycle" step 2). */
helm_status helm_restrict_residual(helm_ctx* ctx, int level, int prec,
                                   const void* u, const void* f, void* rc,
                                   int s);

/* u <- u + P ec (Alg. "Two-grid cycle" step 4), ec on level+1. */
helm_status helm_prolong_add(helm_ctx* ctx, int level, int prec,
                             const void* ec, void* u, int s);

/* u = M_L^{-1} f on the coarsest level (dense inverse times the block):
   FP64 for prec 0, tensor cores (FP16, or three tf32 products: see
   coarse_tf32x3) for prec 1. */
helm_status helm_coarse_solve(helm_ctx* ctx, int prec, const void* f, void* u,
                              int s);

/* z = V-cycle(f) for M (zero initial guess).  f: complex128; z: complex128
   (prec 0) or complex64 (prec 1). */
helm_status helm_vcycle(helm_ctx* ctx, int prec, const void* f, void* z, int s);

/* helm_vcycle without any allocation.  It exists for callers that cannot
   call cudaMalloc at solve time: latency-bound loops that cannot afford the
   device synchronisation an allocation may cause, or frameworks whose
   allocator owns all device memory and forbid others to take more.  Like
   every call here it returns after synchronising the context's stream.
   It computes what helm_vcycle computes (same
   kernels, same arguments and layouts), but its level buffers live in one
   fixed 64 MiB device array compiled into libhelm instead of context
   workspace; every GPU that loads libhelm holds that array until the process
   exits.  The level buffers need 16 (prec 0) or 8 (prec 1) bytes per node
   per column, twice on the fine grid and four times on each coarser grid
   (each rounded up to 256 bytes); prec 1 adds the operands of the
   tensor-core coarsest solve (4 (2 n_c + 31)/32*32 ((2 s + 127)/128*128) bytes
   plus 4 k n_c ((2 s + 127)/128*128) bytes, k the K-split of n_c coarsest
   nodes, at most 16); a call needing more than 64 MiB returns
   HELM_ERR_ARG without touching the GPU.  It calls no cudaMalloc, cudaFree
   or other allocating routine.  The first call on a device looks up the
   array's device address (cudaGetSymbolAddress) with that device current;
   make that first call before any stream capture.  All calls share the
   array and it keeps the last call's contents; calls that overlap on the
   GPU (other streams, other threads on the same device) race, and the
   context must not be used by another thread during the call.  The paper
   has no counterpart of this entry point. */
helm_status helm_vcycle_noalloc(helm_ctx* ctx, int prec, const void* f, void* z, int s);

/* Copy the FP64 stencil of M_level to host: count x K complex128 values,
   K = 9 (2D) or 27 (3D), offset o = sum_k (d_k+1) 3^k for d_k in {-1,0,1}
   along axis k (x1 first); zero where the neighbour is outside the grid.
   Level 0 is returned in the same K-point form. */
helm_status helm_get_operator(const helm_ctx* ctx, int level, void* coef_host);

/* Number of kernels libhelm launched on this context since set-up. */
long long helm_kernel_launches(const helm_ctx* ctx);

/* Orthogonalisation counters of block FGMRES since set-up (see the orth
   field of helm_params): qr = block QR factorisations (one per Krylov step
   and one per restart), reorth = steps whose Gram-Schmidt pass was repeated,
   qr2 = QRs that took a second Cholesky pass.  Any pointer may be NULL.
   HELM_ERR_ARG if ctx is NULL. */
helm_status helm_orth_stats(const helm_ctx* ctx, long long* qr, long long* reorth, long long* qr2);

/* ---------------------------------------------------------------------
 * Learned preconditioning stage (not in the paper; it relies on FGMRES
 * accepting a preconditioner that changes from step to step, Sec. 4).
 * With HELM_MIXED_C64_LEARNED every preconditioner application becomes
 *     z1 = V-cycle(v);  r = v - A z1 (complex64);  rho_j = RMS of column j;
 *     z = z1 + h^2 rho_j N(Re r/rho, Im r/rho, omega^2 m h^2)
 * with N six 3x3 convolutions (ReLU between), 32 hidden channels, BF16
 * weights and activations, FP32 accumulation on the tensor cores; a
 * non-finite network output leaves z1 unchanged.
 * Tensors are NHWC on the 2D node grid: x[b][i][j][c], i the x2 (depth)
 * node index, j the x1 index; weights [co][tap][ci] with tap = 3 dy + dx
 * reading pixel (i + dy - 1, j + dx - 1), zero outside the grid.
 * Weight blob: the bf16 weights of layers 0..5 at byte offsets w_offset,
 * the float biases at b_offset (256-byte aligned), helm_learned_blob_bytes
 * in all.  Channels are padded for the tensor-core tiles: layer 0 reads 16
 * channels (Re r, Im r, kappa, then zeros), layer 5 writes 16 (Re, Im of
 * the correction, then unused).
 * ------------------------------------------------------------------- */
int helm_learned_layers(void);
long long helm_learned_blob_bytes(void);
helm_status helm_learned_layer(int layer, int* cin, int* cout, int* relu, long long* w_offset,
                               long long* b_offset);
/* y[b][i][j][co] = epilogue(bias[co] + sum_{tap, ci} w[co][tap][ci] x[b][..][ci]);
   epilogue: ReLU if relu, then zero where mask (bf16, cout channels, may be
   NULL) is not > 0; y bf16, or float if y_float.  (cin, cout) in {(16,32),
   (32,32), (32,16), (16,16)}.  All device pointers; enqueued on stream and
   synchronised.  The data gradient of a layer is this call with the weights
   from helm_conv3x3_flip and the layer below's activation as the mask. */
helm_status helm_conv3x3(const void* x, int batch, int H, int W, int cin, const void* w,
                         const float* bias, int cout, int relu, const void* mask, void* y,
                         int y_float, void* stream);
/* dw[co][tap][ci] += sum over pixels gy[co] x[shifted][ci]; db[co] += sum gy[co]
   (FP32 accumulators, caller zeroes them). */
helm_status helm_conv3x3_wgrad(const void* x, const void* gy, int batch, int H, int W, int cin,
                               int cout, float* dw, float* db, void* stream);
/* wf[ci][tap][co] = w[co][8 - tap][ci] for ci < cin, zero for cin <= ci < cin_out. */
helm_status helm_conv3x3_flip(const void* w, int cin, int cout, void* wf, int cin_out, void* stream);
/* Adam step (bias-corrected, step >= 1) on FP32 parameters p with gradient g and
   moments m, v; p_bf16 (may be NULL) receives the bf16 copy. */
helm_status helm_adam(float* p, const float* g, float* m, float* v, void* p_bf16, int n, float lr,
                      float b1, float b2, float eps, int step, void* stream);
/* Network input for a block: r = f - A z (f complex128, z complex64, internal
   layout, N x s), rho_out[j] = RMS of column j of r, x_out = bf16 NHWC
   [s][N2][N1][16].  Allocates its own temporaries. */
helm_status helm_learned_input(helm_ctx* ctx, const void* f, const void* z, int s, void* x_out,
                               float* rho_out);
/* Residual-loss training inputs for a block (not in the paper; the loss of
   helm_learned_residual_loss): as helm_learned_input, plus, per sample j in
   NHWC image order [s][N2][N1], r_out = r / rho_j and coef_out = h^2 c_A =
   kappa (1 - i gamma), both as float pairs (re, im).  Allocates its own
   temporaries. */
helm_status helm_learned_residual_input(helm_ctx* ctx, const void* f, const void* z, int s, void* x_out,
                                        float* rho_out, float* r_out, float* coef_out);
/* Residual of the corrected iterate as the training loss (not in the paper):
   with e_b = pred_b channels (0, 1) as a complex image and K = h^2 A on the
   image grid (K e = 4 e - the four neighbours (zero outside) - coef e),
       q_b = r_b - K e_b,   loss = mean_b ||q_b||^2 / ||r_b||^2,
   grad (bf16 [B][H][W][16], channels 0, 1) = -(2 / (B ||r_b||^2)) K^H q_b
   (K^H uses conj(coef)).  pred: float [B][H][W][16]; r, coef: float pairs
   [B][H][W]; q: float-pair scratch [B][H][W]; sums: 2B floats of scratch;
   loss_out: device float.  All device pointers; enqueued on stream and
   synchronised. */
helm_status helm_learned_residual_loss(const float* pred, const float* r, const float* coef, int batch, int H,
                                       int W, float* q, float* sums, void* grad, float* loss_out,
                                       void* stream);
/* v[node][j] = r[j][node] as complex128: an image-order block of float pairs
   [s][N] to the internal layout (the next vector of a training chain). */
helm_status helm_learned_image_to_block(const float* r, long long N, int s, void* v, void* stream);
/* Training target t[j][node][0..1] = scale * e[node][j] / rho[j] (e complex64,
   internal layout); scale = 1/h^2 makes it the network's output units. */
helm_status helm_learned_target(const void* e, long long N, int s, const float* rho, float scale,
                                float* t_out, void* stream);
/* loss = mean_b ||pred_b - t_b||^2 / ||t_b||^2 (pred: float [B][P][16], channels
   0, 1 used; t: float [B][P][2]); grad: bf16 [B][P][16]; sums: 2B floats of
   scratch; loss_out: device float. */
helm_status helm_learned_loss(const float* pred, const float* t, int batch, long long P, float* sums,
                              void* grad, float* loss_out, void* stream);

/* ---------------------------------------------------------------------
 * FWI sensitivities (Sec. 2.4 Eq. fwisens; data Eq. data; misfit Eq. minp
 * without regularisation).  In this library's sign convention
 *     J = du/dm = w^2 A^{-1} diag((1 - i g) u),
 * data are the fields sampled at receiver nodes recv (device int array of
 * nrec node indices), and for real m
 *     J^T w = sum over sources Re(conj(w^2 (1 - i g) u_j) lambda_j),
 *     lambda_j = A^{-H} P w_j  (one adjoint solve per source).
 * Fields U: device, ABI layout (s x N), complex128, or 16-bit pairs
 * (half re, half im; fields_half = 1), the storage Sec. 2.4 uses for the
 * forward fields.  Data blocks (W, d_obs, jv output): device complex128,
 * s x nrec (column j = source j).  Solves use the context's solver and tol;
 * each call allocates its temporaries (HELM_ERR_NOMEM if it cannot; nothing
 * is kept).  Receiver indices must lie in [0, N): each call copies the nrec
 * indices to the host and returns HELM_ERR_ARG, before any kernel runs, if
 * one does not.
 * ------------------------------------------------------------------- */
/* U16[e] = (half) U[e] for N*s complex values. */
helm_status helm_fields_to_half(const void* U, long long N, int s, void* U16, void* stream);
/* out = P^T J v per source (v: device double[N]). */
helm_status helm_fwi_jv(helm_ctx* ctx, const void* fields, int fields_half, int s, const double* v,
                        const int* recv, int nrec, double tol, void* out);
/* out[k] = (J^T w)_k summed over the s sources (device double[N]). */
helm_status helm_fwi_jtw(helm_ctx* ctx, const void* fields, int fields_half, int s, const void* W,
                         const int* recv, int nrec, double tol, double* out);
/* Forward solve of Q, data residual U[recv] - d_obs, misfit (host, may be
   NULL) = 1/2 sum |residual|^2, gradient grad = J^T residual (device
   double[N]); store_half keeps the forward fields in 16 bits for the
   gradient product; U_out (device, may be NULL) receives the fields. */
helm_status helm_fwi_gradient(helm_ctx* ctx, const void* Q, int s, const void* d_obs, const int* recv,
                              int nrec, double tol, int store_half, double* grad, double* misfit,
                              void* U_out);

/* ---------------------------------------------------------------------
 * Per-kernel profiler (the per-RHS timing of Sec. 5.3's table, broken down
 * by kernel).  When enabled, every launch on the context is bracketed by a
 * CUDA event pair on the context's stream and tagged with its algorithmic
 * bytes and flops (each vector element read or written once, coefficients
 * once per node).  Enabling resets the totals; disabling frees the events.
 * ------------------------------------------------------------------- */
helm_status helm_profile_enable(helm_ctx* ctx, int enable);
/* While the profiler is enabled, record only launches of class kid (their
   event pairs, bytes and flops); -1 records every class (the state after
   helm_profile_enable).  HELM_ERR_ARG if the profiler is off or kid is out
   of range.  Fewer events in flight perturb the timed work less. */
helm_status helm_profile_select(helm_ctx* ctx, int kid);
/* Number of kernel classes and the name of class kid (static strings). */
int helm_profile_kernel_count(void);
const char* helm_profile_kernel_name(int kid);
/* Totals of class kid since enabling: summed event time (ms), launches,
   algorithmic bytes and flops.  Synchronises the context's stream. */
helm_status helm_profile_read(helm_ctx* ctx, int kid, double* time_ms, long long* launches,
                              double* bytes, double* flops);

/* ---------------------------------------------------------------------
 * Factored eikonal equation and its sensitivities (Sec. 2.5: Eq.
 * factoredeikonal discretised by the first-order factored upwind scheme of
 * Eq. Gudonov / Eq. FOfactoredD, solved by the fast marching algorithm;
 * sensitivities by Eq. Sensitivity / Sensitivity2).  tau = tau0 tau1 with
 * tau0 = |x - x_s|; m is the squared slowness (the Helmholtz m) on the same
 * node grid: (n[k] + 1) nodes per axis, x1 fastest.  One fast marching per
 * source (ordering: least tau0 tau1 first, ties by node index); the local
 * solve is the Godunov equation solved exactly from accepted neighbours (the
 * least root consistent with the max{}); the source node holds
 * tau1 = sqrt(m_s).  The workspace keeps, per source, tau1 in single
 * precision, the chosen derivative per node and the fast-marching wavefront
 * levels, from which J v and J^T w are applied by forward / backward
 * substitution in fast-marching order (Eq. Sensitivity2 is lower triangular
 * in that order).  All calls run on the workspace's stream and return after
 * synchronising it.
 * ------------------------------------------------------------------- */
typedef struct helm_eik helm_eik;

/* Workspace for up to ns_max sources on a dim-dimensional grid of n[k] cells
   per axis (x1, x2[, x3]) with spacing h (metres).  Device memory: about
   (46 N + 16) bytes per source, N = number of nodes.  HELM_ERR_ARG on bad
   sizes, HELM_ERR_NOMEM when the allocation fails. */
helm_status helm_eik_create(int dim, const int* n, double h, int ns_max, void* cuda_stream,
                            helm_eik** out);
/* Fast marching for ns <= ns_max sources.  m: device, N doubles (positive).
   src: host, ns x dim node indices (x1, x2[, x3]) per source, inside the
   grid.  Optional device outputs (NULL to skip), each ns x N, source-major:
   tau_out (travel time tau0 tau1, FP64), tau1_out (FP64), order_out (node of
   each acceptance step, int32), dir_out (per node: 2 bits per axis from the
   slowest axis (x3 in 3D, x2 in 2D) in the low bits, 1 backward / 2 forward
   derivative, 0xFF at the source).  HELM_ERR_NOMEM if a heap would overflow
   (not met on a connected grid), HELM_ERR_BREAKDOWN if a node is unreached. */
helm_status helm_eik_forward(helm_eik* e, const double* m, const int* src, int ns, double* tau_out,
                             double* tau1_out, int* order_out, unsigned char* dir_out);
/* z (device, ns x N) = J_s v for every source of the last forward call,
   J_s = d tau1 / d m (Eq. Sensitivity), v: device, N doubles. */
helm_status helm_eik_jv(helm_eik* e, const double* v, double* z);
/* y (device, ns x N) = J_s^T w_s, w: device, ns x N doubles. */
helm_status helm_eik_jtw(helm_eik* e, const double* w, double* y);
/* Last error message of the workspace ("" if none). */
const char* helm_eik_last_error(const helm_eik* e);
void helm_eik_destroy(helm_eik* e);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
