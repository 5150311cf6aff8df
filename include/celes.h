/*
 * celes.h -- C ABI of the GB300 (sm_103a) multi-sphere T-matrix solver.
 *
 * The library solves the master equation of the multiple-scattering problem
 * (CELES, JQSRT 2017, Sec. 2.2, Eqs. for a^i, M and the master equation):
 *
 *     sum_{i',n'} M^{ii'}_{nn'} b^{i'}_{n'} = sum_{n'} T^i_{nn'} a^i_{in,n'},
 *     M^{ii'}_{nn'} = delta_{nn'} delta_{ii'} - sum_{n''} T^i_{nn''} W^{ii'}_{n''n'},
 *     W^{ii'}_{nn'} = A_{n'n}(r_i - r_i')           (App. A.2 translation operator)
 *
 * with an iterative solver whose matrix-vector products evaluate the coupling
 * blocks on the fly (Sec. 3.2).  All compute runs in CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lengths in one user-chosen unit (the tests use nanometres); k0 = 2 pi /
 *    lambda_vacuum in the inverse unit.  Background wavenumber k = n0 k0.
 *  - Coefficient order per sphere (fixed by this library; the paper fixes
 *    none): n = (tau-1) L(L+2) + l(l+1) - 1 + m, tau in {1,2}, l = 1..L,
 *    m = -l..l; nmax = 2 L (L+2).
 *  - Complex numbers are interleaved (re, im).  FP64 data are complex128,
 *    FP32 data complex64.  Coefficient vectors are [nrhs][N][nmax].
 *  - Host pointers are only read during the call; the library copies what it
 *    keeps.  Device pointers passed to the *_matvec / *_apply calls belong to
 *    the caller and must hold the stated number of elements on the context's
 *    device; the library never frees them.
 *  - stream: a cudaStream_t passed as void*; NULL means the context's own
 *    stream.  Calls taking a stream are stream-ordered and do not synchronise.
 *  - Every call returns a celes_status; on failure celes_last_error() gives a
 *    one-line reason.  Invalid arguments return CELES_EINVAL before any GPU
 *    work is queued.
 */
#ifndef CELES_H_
#define CELES_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct celes_ctx celes_ctx;

typedef enum {
  CELES_OK = 0,
  CELES_EINVAL = -1,    /* invalid argument */
  CELES_ENOMEM = -2,    /* device allocation failed */
  CELES_ECUDA = -3,     /* CUDA runtime error */
  CELES_ENOCONV = -4,   /* solver stopped before the tolerance; best iterate kept */
  CELES_ENUMERIC = -5,  /* NaN/Inf or breakdown detected */
  CELES_EOVERLAP = -6,  /* two spheres overlap (|r_i - r_j| < R_i + R_j) */
  CELES_ETIMEOUT = -7,  /* a bounded device wait gave up */
  CELES_ESTATE = -8,    /* call out of order (e.g. solve before set_incident) */
  CELES_ETOOBIG = -9    /* problem larger than a fixed-size buffer allows */
} celes_status;

typedef enum { CELES_FP64 = 0, CELES_FP32 = 1 } celes_precision;

typedef enum {
  CELES_KERNEL_AUTO = 0,    /* rotation-translation-rotation in both precisions */
  CELES_KERNEL_DIRECT = 1,  /* per-entry evaluation of W^{ij} (App. A.2 formula as printed) */
  CELES_KERNEL_RTR = 2      /* W = D^H W_z D (rotation, axial translation, rotation), both precisions */
} celes_kernel;

typedef struct {
  int device;           /* CUDA device ordinal (default 0) */
  int check_overlap;    /* reject overlapping spheres (default 1) */
  int chunks;           /* source chunks of the coupling kernel; 0 = automatic */
  int kernel;           /* celes_kernel: coupling-kernel variant (default AUTO) */
  int autotune;         /* 1 (default): the first FP32 coupling product times the candidate launch
                           shapes and source-chunk counts of the coupling kernel on this problem
                           (cached per device, lmax and size class) and keeps the fastest; it
                           synchronises, so make that first product before any stream capture.
                           0 (and FP64 always): the built-in shape, about eight waves of chunks */
  int variant;          /* -1 (default): as autotune decides; 0..7 force the launch shape: bit 0 the
                           FP32 compile-time shape (0 = built-in, 1 = the alternative; FP64 always
                           uses the built-in one), bit 1 the cluster reduction of the partial sums
                           (thread-block clusters of up to 8 source chunks), bit 2 (FP32 only) the
                           partial sums of all chunks added into one slice by vector reductions in
                           L2, so that only the final sums reach DRAM; with bit 2 the summation
                           order, and so the last bits of an FP32 product, vary between calls.
                           Values above 7 give CELES_EINVAL */
} celes_options;

typedef enum { CELES_PLANE_WAVE = 0, CELES_GAUSSIAN_BEAM = 1 } celes_incident_kind;

/* One incident field (one right-hand side).
 *  Plane wave (App. A.1 PVWF): E = E0 Phi_pol(alpha, beta; r), pol 1 = along
 *    e_alpha, 2 = along e_beta.  beta = 0, alpha = 0, pol = 2 is x-polarised
 *    along +z.
 *  Gaussian beam (App. C): waist w, focus r_G, polarisation
 *    E0 (-sin alpha_G e_x + cos alpha_G e_y), angular spectrum restricted to
 *    beta in [0, pi/2]; n_beta Gauss-Legendre nodes (0 = 128). */
typedef struct {
  int kind;
  double beta, alpha;
  int pol;
  double E0_re, E0_im;
  double waist;
  double focus[3];
  double alpha_G;
  int n_beta;
} celes_incident;

typedef enum {
  CELES_SOLVE_FP64 = 0,   /* plain FP64 GMRES, FP64 coupling matvec */
  CELES_SOLVE_MIXED = 1   /* FP32 inner GMRES + FP64 residual refinement */
} celes_solve_mode;

typedef enum {
  CELES_X0_TA = 0,     /* initial guess T a_in */
  CELES_X0_USER = 1,   /* guess given by celes_set_initial_guess */
  CELES_X0_ZERO = 2,
  CELES_X0_LEARNED = 3 /* guess from celes_gnn_predict, used only where its residual is below that of T a_in */
} celes_x0_kind;

typedef enum {
  CELES_SOLVER_GMRES = 0,    /* restarted GMRES, classical Gram-Schmidt twice (Sec. 3.2) */
  CELES_SOLVER_BICGSTAB = 1  /* BiCGSTAB (van der Vorst), the other Krylov solver named in Sec. 3.2 */
} celes_solver;

typedef struct {
  int mode;             /* celes_solve_mode */
  int restart;          /* GMRES restart length (default 100) */
  int max_iter;         /* total inner iterations (default 2000) */
  int max_outer;        /* refinement steps in MIXED mode (default 20) */
  int x0;               /* celes_x0_kind */
  int use_precond;      /* apply the block preconditioner if built (default 1) */
  double inner_tol;     /* MIXED: relative tolerance floor of each FP32 solve (default 1e-5) */
  int solver;           /* celes_solver (default GMRES; restart is ignored by BiCGSTAB) */
} celes_solve_opts;

typedef struct {
  int status;               /* celes_status of the solve */
  int iterations;           /* total GMRES iterations (all precisions) */
  int outer;                /* refinement steps (MIXED) or restarts (FP64) */
  int matvecs_fp64;         /* coupling matvecs in FP64 */
  int matvecs_fp32;         /* coupling matvecs in FP32 */
  double residual;          /* final ||T a - M b|| / ||T a||, FP64, per RHS max */
  double seconds;           /* wall time of the solve */
  double* history;          /* optional caller buffer for the residual history */
  int history_cap;          /* its capacity */
  int history_len;          /* entries written */
  int guess_used;           /* RHS that started from the user / learned guess */
} celes_solve_info;

/* Create a context: copies positions [N][3], radii [N] and the complex
 * refractive indices n_i [N] (re, im pairs) to the device, validates them and
 * computes the Mie T-matrix (App. B) in FP64 on the GPU.
 * lmax in 1..5.  opt may be NULL (defaults).  On success *out owns all device
 * memory of the problem; release it with celes_destroy. */
int celes_create(celes_ctx** out, int64_t N, const double* positions, const double* radii, const double* n_i,
                 double n0, double k0, int lmax, const celes_options* opt);

/* Set nrhs incident fields (array of nrhs descriptors) and compute their
 * coefficients a_in (App. A.2 PVWF->SVWF transform for plane waves, App. C
 * beta quadrature for Gaussian beams) in FP64 on the GPU.  Resets any
 * previous solution. */
int celes_set_incident(celes_ctx* ctx, const celes_incident* inc, int nrhs);

/* y = W x (Sec. 2.2, Sec. 3.2.2): y_i = sum_{j != i} W^{ij} x_j for nrhs
 * vectors, blocks evaluated on the fly.  x, y: device pointers to
 * [nrhs][N][nmax] complex128 (CELES_FP64) or complex64 (CELES_FP32); x and y
 * must not overlap. */
int celes_coupling_matvec(celes_ctx* ctx, const void* x, void* y, int nrhs, int precision, void* stream);

/* y = M x = x - T (W x) (Sec. 2.2, Eq. for M): the coupling matvec with the
 * T-matrix epilogue fused (Sec. 3.2.2).  Same layout rules as above. */
int celes_master_matvec(celes_ctx* ctx, const void* x, void* y, int nrhs, int precision, void* stream);

/* Build the block-diagonal preconditioner (Sec. 3.2.1): partition the
 * spheres by cuboids of the given edge (grid anchored at the minimum corner of
 * the centres' bounding box, cuboids ordered by (z, y, x) index), assemble
 * each diagonal block of M in FP64 and LU-factor it with partial pivoting on
 * the GPU.  Replaces any earlier preconditioner. */
int celes_precond_build(celes_ctx* ctx, double cuboid_edge);

/* Launch shape the context's coupling kernel uses in `precision`: variant
 * (bit 0: alternative FP32 shape; bit 1: cluster reduction of the partial
 * sums; bit 2: reduction in L2, see celes_options.variant), source chunks
 * per product and, if
 * the autotuner chose it, the timed duration of the winning candidate (ms; 0
 * otherwise).  CELES_ESTATE before the first coupling product in that
 * precision.  Measurement support; the paper has no counterpart. */
int celes_coupling_shape(const celes_ctx* ctx, int precision, int* variant, int* chunks, double* ms);

/* Size of the built block preconditioner: number of blocks (cuboids that
 * hold spheres), largest block dimension (unknowns) and the total number of
 * complex entries of all blocks' factors (the apply reads each once: 16 bytes
 * per entry for FP64 vectors, 8 for FP32).  CELES_ESTATE before a build.
 * Measurement support; the paper has no counterpart. */
int celes_precond_stats(const celes_ctx* ctx, int64_t* nblocks, int64_t* max_dim, int64_t* entries);

/* y = P^{-1} x with P the block-diagonal part of M (Sec. 3.2.1, step 4):
 * per block, solve L_j U_j y = P_j x.  Layout as for the matvecs.  FP64
 * vectors use the FP64 factors; FP32 vectors an FP32 copy of them made at
 * build time (the same operator wherever the FP32 solver applies it).  x and
 * y may be equal. */
int celes_precond_apply(celes_ctx* ctx, const void* x, void* y, int nrhs, int precision, void* stream);

/* Provide an initial guess b0 ([nrhs][N][nmax] complex128, host) used by
 * celes_solve with x0 = CELES_X0_USER (Sec. 4.2, custom initial condition). */
int celes_set_initial_guess(celes_ctx* ctx, const double* b0_host);

/* Solve M b = T a_in for every RHS to ||T a - M b|| / ||T a|| <= tol
 * (FP64 residual).  o and info may be NULL.  Returns CELES_ENOCONV if the
 * iteration budget ran out (the best b is still stored), CELES_ENUMERIC if a
 * residual or Krylov vector norm is not finite (e.g. a NaN user guess) or
 * GMRES meets a singular Hessenberg matrix; b is then not meaningful. */
int celes_solve(celes_ctx* ctx, double tol, const celes_solve_opts* o, celes_solve_info* info);

/* Copy results to the host ([nrhs][N][nmax] complex128). */
int celes_get_coefficients(celes_ctx* ctx, double* b_host);
int celes_get_incident_coefficients(celes_ctx* ctx, double* a_host);
/* T-matrix diagonal: [N][nmax] complex128 in coefficient order. */
int celes_get_tmatrix(celes_ctx* ctx, double* t_host);

/* Plane-wave amplitude of the scattered field of RHS `rhs` (App. D):
 *   g_j(alpha, beta) = 1/(2 pi) sum_i e^{-i k.r_i} sum_n B_nj(beta) e^{i m alpha} b^i_n
 * for Nd directions dirs [Nd][2] = (beta, alpha); writes g [Nd][2] complex128
 * (host).  The radiant intensity is 2 pi^2/(omega k mu0) |g_j|^2. */
int celes_farfield(celes_ctx* ctx, const double* dirs, int64_t Nd, double* g, int rhs);

/* Electric field at Np points (Sec. 2.1), FP64, RHS `rhs`:
 *   what = 0: scattered field sum_i sum_n b^i_n Psi^(3)_n(r - r_i) (needs a
 *             solution), 1: incident field (plane wave App. A.1, or the
 *             Gaussian beam's angular spectrum of App. C with the same beta
 *             nodes as its coefficients), 2: their sum.
 * points [Np][3] and E [Np][3] complex128 are host arrays.  Points inside a
 * sphere get NaN for what = 0 and 2 (the internal field is not computed).
 * Errors: EINVAL, ESTATE (no incident field, or no solution for what != 1),
 * ENOMEM, ECUDA. */
int celes_nearfield(celes_ctx* ctx, const double* points, int64_t Np, int rhs, int what, double* E);

/* Reflected and transmitted power fractions R, T of RHS `rhs` (App. D; the
 * reflectivity and transmittivity of Sec. 4): T = forward-hemisphere flux of
 * the total field, R = backward-hemisphere flux of the scattered field, both
 * divided by the Gaussian beam's power.  Quadrature: n_beta Gauss-Legendre
 * nodes in beta per hemisphere, n_alpha trapezoid nodes in alpha.  Needs a
 * solution and a Gaussian-beam RHS (EINVAL for a plane wave, whose power is
 * not finite).  For lossless spheres R + T = 1 up to truncation and
 * quadrature error. */
int celes_power(celes_ctx* ctx, int rhs, int n_beta, int n_alpha, double* R, double* T);

/* Phase-matrix element S11 (Sec. 4: the average of a TE and a TM run's
 * far-field intensity): s11[i] = (1/2) sum over the two RHS rhs_a, rhs_b of
 * the azimuthal mean (n_alpha trapezoid nodes) of sum_j |g_j(alpha, beta_i)|^2
 * (App. D), for n_beta polar angles betas (host); unnormalised (divide by the
 * forward value for S11(0) = 1).  Needs a solution.  Errors: EINVAL, ESTATE,
 * ENOMEM, ECUDA. */
int celes_s11(celes_ctx* ctx, int rhs_a, int rhs_b, const double* betas, int n_beta, int n_alpha, double* s11);

/* Problem sizes. */
int64_t celes_num_spheres(const celes_ctx* ctx);
int celes_nmax(const celes_ctx* ctx);
int celes_num_rhs(const celes_ctx* ctx);

/* Number of nonzero (a5, b5) terms of the coupling block built into the
 * kernels for degree lmax (App. A.2), and their values: for every term t,
 * idx[5t..5t+4] = (source row, receiving row, p, mu, kind) with rows
 * r = l(l+1) - 1 + m, kind 0 = a5 (real) and 1 = b5/i (real), val[t] its
 * real factor.  Host-only; pass NULL buffers to query the count.  Returns the
 * count (>= 0) or CELES_EINVAL. */
int celes_coupling_terms(int lmax, int* idx, double* val, int cap);

/* Kernel timing with CUDA events recorded on the stream each kernel is
 * launched on.  celes_profile(ctx, 1) starts recording (and clears earlier
 * records), 0 stops.  celes_kernel_time(ctx, which, &ms, &launches)
 * synchronises the context's stream and returns the summed duration and the
 * launch count of one kernel class: which = 0 FP32 coupling kernel, 1 FP64
 * coupling kernel, 2 coupling epilogue (both precisions).  The paper has no
 * counterpart; this is measurement support. */
int celes_profile(celes_ctx* ctx, int on);
int celes_kernel_time(celes_ctx* ctx, int which, double* ms, int64_t* launches);

/* Number of kernels this library has launched in the process so far. */
int64_t celes_kernel_launches(void);

/* Algorithmic flops per ordered sphere pair and right-hand side of the
 * coupling matvec for degree lmax and kernel variant (celes_kernel): the
 * direct per-entry evaluation counts 4 (a5 + b5 terms) + 12 NH^2 + 2 NS + 4
 * nmax^2; the rotation-translation-rotation variant counts its own rotations,
 * Wigner-d sums, axial build/apply and phases.  Host-only; -1 on bad lmax. */
double celes_flops_per_pair(int lmax, int kernel);

/* Measured fused multiply-add issue peak of the current device, the
 * denominator of the coupling kernels' roofline (the paper has no
 * counterpart; this is measurement support).  kind: 0 = FP64 FMA, 1 = FP32
 * FMA, 2 = FP32 packed two-lane FMA (sm_100 and later).  Every thread of a
 * 4 x 256-thread-per-SM grid runs 16 independent FMA chains; the best of three
 * CUDA-event-timed launches gives *tflops (2 flops per FMA) and *ms.  The
 * figure holds at the SM clock of that moment; sample the clock beside it.
 * Allocates a small output buffer, synchronises. */
int celes_fma_peak(int kind, double* tflops, double* ms);

/* Tensor-core GEMM C = alpha A B^T + beta C (the dense layers of the learned
 * initial guess; the paper has no counterpart).  A: [M][K] BF16, B: [N][K]
 * BF16 (row-major, K contiguous, lda/ldb in elements), C: [M][N] FP32
 * (row-major, ldc).  Device pointers; K, lda, ldb multiples of 8 and A, B
 * 16-byte aligned (else CELES_EINVAL).  Runs tcgen05.mma (kind::f16, FP32
 * accumulation in tensor memory) on sm_103a; synchronises the stream and
 * returns CELES_ETIMEOUT if a bounded wait on the tensor core gave up. */
int celes_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc, float alpha,
                    float beta, void* stream);

/* Learned initial guess (Sec. 4.2: the solver accepts a custom initial
 * condition).  A graph network over each sphere's 16 nearest neighbours
 * (relative positions in wavelengths, k R_i, n_i, the scaled T a_in of the
 * sphere) predicts d_i = b_i - (T a_in)_i; the first iterate is T a_in + d.
 * Layers: input 1 dense, `layers` message-passing rounds (message MLP on
 * [h_j; h_i; e_ij], mean aggregation, residual update MLP), output dense; all
 * dense layers run on the tcgen05 BF16 GEMM with FP32 accumulation, and
 * training (MSE, Adam) uses hand-written backward kernels.
 *   celes_gnn_create : width (multiple of 16, <= 512), layers (1..8), knn = 16;
 *                      the output layer starts at zero (untrained guess = T a)
 *   celes_gnn_train  : `steps` Adam steps on one solved context (its current
 *                      solution b of RHS `rhs` is the target); loss_out gets
 *                      the last MSE (scaled units); CELES_ESTATE if unsolved
 *   celes_gnn_predict: computes the guess for every RHS of a context and
 *                      stores it for celes_solve with x0 = CELES_X0_LEARNED
 * The paper has no counterpart of the network itself; the final FP64 residual
 * of the solve decides whether it helped, and celes_solve falls back to
 * T a_in per RHS when its residual is not smaller. */
typedef struct celes_gnn celes_gnn;
int celes_gnn_create(celes_gnn** out, int lmax, int width, int layers, int knn, uint64_t seed, int device);
int celes_gnn_train(celes_gnn* g, celes_ctx* ctx, int rhs, int steps, double lr, double* loss_out);
int celes_gnn_predict(celes_gnn* g, celes_ctx* ctx);
/* Training over many ensembles without keeping their contexts:
 *   celes_gnn_add_example  : copies a solved context's graph (16-NN lists),
 *                            node and edge features and target (b - T a) of
 *                            RHS `rhs` into the network's own device memory
 *                            (about 1 KB per sphere) and returns its index in
 *                            *idx; the context may then be destroyed;
 *                            CELES_ESTATE if unsolved
 *   celes_gnn_train_example: `steps` Adam steps on stored example idx
 *                            (steps = 0: loss only); loss_out as in train
 *   celes_gnn_num_examples / celes_gnn_clear_examples: count / free them. */
int celes_gnn_add_example(celes_gnn* g, celes_ctx* ctx, int rhs, int* idx);
int celes_gnn_train_example(celes_gnn* g, int idx, int steps, double lr, double* loss_out);
int celes_gnn_num_examples(const celes_gnn* g);
int celes_gnn_clear_examples(celes_gnn* g);
int celes_gnn_num_params(const celes_gnn* g);
/* Copy the parameters (what = 0) or the gradients of the last training pass
 * (what = 1) to `host` as FP32, layer by layer (input, then message and update
 * of each round, then output), each layer as its weight [out][in] row-major
 * followed by its bias [out].  host = NULL returns the count.  celes_gnn_train
 * with steps = 0 computes the loss and gradients without updating. */
int celes_gnn_export(celes_gnn* g, int what, float* host, int cap);
void celes_gnn_destroy(celes_gnn* g);

/* Coupling matvec y = W x that allocates no device memory (the paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: code running under a host application's own device-memory pool,
 * where direct allocations are forbidden, and latency-critical code that
 * cannot afford the device-wide synchronisation of cudaMalloc/cudaFree).
 * It needs no context: the caller passes everything in its own device memory.
 *   positions4 : device pointer to [N][4] doubles (x, y, z, unused), 32-byte
 *                aligned
 *   k          : background wavenumber n0 * k0
 *   x, y       : device pointers to [N][nmax] complex128 (CELES_FP64) or
 *                complex64 (CELES_FP32); one right-hand side; must not overlap
 *   stream     : cudaStream_t as void* (NULL = the default stream)
 * The kernel's scratch (its per-chunk partial sums) lives in one static
 * 32 MiB device array compiled into the library, which every GPU that loads
 * the library holds until the process exits.  Sizes whose single partial sum
 * N * nmax * (16 or 8 bytes) exceeds 32 MiB return CELES_ETOOBIG before any GPU
 * work (e.g. lmax 4: N <= 87381 in FP32, N <= 43690 in FP64).  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * and sets the kernel's shared-memory attribute; make that first call before
 * any stream capture.  The array holds the previous call's partial sums; every
 * call overwrites all of the part it reads, so nothing needs clearing.  All
 * calls share the one array, so calls that overlap on the GPU (other streams,
 * other host threads) race: serialise them.  Stream ordered, no
 * synchronisation; uses the rotation-translation-rotation kernel. */
int celes_coupling_matvec_noalloc(int64_t N, int lmax, double k, const double* positions4, const void* x, void* y,
                                  int precision, void* stream);

void celes_destroy(celes_ctx* ctx);
const char* celes_last_error(const celes_ctx* ctx);

/* ---- Batched solves over many ensembles (multi-RHS, uneven sizes) --------
 * A batch groups contexts (same device, any lmax and N, incident fields set)
 * and solves the master equation (I - T W) b = T a_in (Sec. 2.2) for every
 * right-hand side of every context in lockstep: the coupling products of all
 * systems of one lmax run as one persistent launch that balances tiles of all
 * ensembles, the operator is replayed from a CUDA graph, and the Krylov
 * vector work of all systems runs in segmented kernels with one host
 * synchronisation per Gram-Schmidt stage for the whole batch.
 *
 * celes_batch_create: ctxs [count] stay owned by the caller and must outlive
 *   the batch; restart is the GMRES restart length (<= 0: 30).  Copies T a of
 *   every system.  Errors: EINVAL (bad arguments, contexts on different
 *   devices), ESTATE (a context without incident field), ENOMEM.
 * celes_batch_master_matvec: y = (I - T W) x on the flat vectors of the
 *   batch (device pointers; systems concatenated in context order, RHS-major
 *   inside a context, [N][nmax] complex each; complex128 for FP64, complex64
 *   for FP32).  Synchronous.
 * celes_batch_solve: GMRES per system (no preconditioner, first iterate
 *   T a), MIXED (FP32 inner + FP64 refinement) or FP64, to
 *   ||T a - M b|| / ||T a|| <= tol per system; writes b into each context
 *   (read with celes_get_coefficients) and infos [count] (per context: max
 *   over its RHS; residual history not recorded).  opts may be NULL; its
 *   x0 must be CELES_X0_TA and its solver GMRES; use_precond is ignored.
 *   Returns OK, ENOCONV (some system missed tol; b still written), ENUMERIC,
 *   ECUDA. */
typedef struct celes_batch celes_batch;
int celes_batch_create(celes_batch** out, celes_ctx* const* ctxs, int count, int restart);
int celes_batch_num_systems(const celes_batch* b);
long long celes_batch_num_unknowns(const celes_batch* b);
int celes_batch_master_matvec(celes_batch* b, const void* x, void* y, int precision);
int celes_batch_solve(celes_batch* b, double tol, const celes_solve_opts* opts, celes_solve_info* infos);
const char* celes_batch_last_error(const celes_batch* b);
void celes_batch_destroy(celes_batch* b);

const char* celes_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CELES_H_ */
