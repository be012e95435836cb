/*
 * adp.h -- C ABI of libadp.so, the GB300 (sm_103a) hot path of ADP-beta solved
 * by the Method of Adaptive Inexact Descent (MAID), arXiv 2502.09758.
 *
 * Problem (Eq. 2.5 with the finite-dimensional instantiation of Sec. 3.2):
 *
 *   min_b  ell(b) = g(x^(b)) + r(b),   x^(b) = argmin_x h(x, b)
 *   h(x, b) = 1/2 ||B x - y||^2 + alpha J(x)       (lower level, Eq. 2.5b)
 *   g(x)    = ||A x - y||^2                          (upper fidelity)
 *   r(b)    = beta (w0 ||b-a||^2 + ||D_h(b-a)||^2 + ||D_v(b-a)||^2)   (Sobolev, Sec. 4.2)
 *
 * B x is the discrete integral operator T(b, x) of Eq. 2.4: a centred periodic
 * convolution per channel, (B x)[c,i,j] = sum_{p,q} b[c,p,q] x[c,i-p+r,j-q+r]
 * with r = (K-1)/2 and indices taken modulo H and W.  A is the same operator
 * with the fixed kernel a.  J is an anisotropic smoothed total variation,
 * J(x) = sum phi((D_h x)) + phi((D_v x)) with periodic forward differences.
 *
 * Layouts: images are planar C x H x W, row-major, contiguous; kernels are
 * C x K x K, row-major, contiguous.  Element type: float for ADP_F32, double
 * for ADP_F64 (the `prec` of the problem); every `void*` data argument below
 * has that type.  All data pointers are DEVICE pointers on the problem's
 * device, owned by the caller; the library reads inputs and writes only the
 * outputs named on each call, and never frees caller memory.
 *
 * Execution: every call is ordered on the stream given at creation, launches
 * one cooperative kernel, and returns after that stream has finished the call
 * (scalar outputs are valid on return).  Calls on one problem must not run
 * concurrently.  No C++ exception crosses this boundary.  Every device-side
 * wait is bounded by `wait_timeout_s`; a wait that gives up returns
 * ADP_ETIMEOUT and leaves the CUDA context usable.
 */
#ifndef ADP_H
#define ADP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ADP_OK = 0,
    ADP_EINVAL = 1,      /* bad argument (null pointer, size, unsupported K)      */
    ADP_ENOMEM = 2,      /* workspace allocation failed                            */
    ADP_ECUDA = 3,       /* CUDA runtime error (message in adp_last_error)          */
    ADP_ENONFINITE = 4,  /* a NaN/Inf appeared in a norm or a dot product           */
    ADP_ENOCONV = 5,     /* an iterative solve hit its cap; outputs are valid       */
    ADP_ELSFAIL = 6,     /* MAID backtracking rounds exhausted; b unchanged         */
    ADP_ETIMEOUT = 7     /* a bounded device-side wait gave up                      */
} adp_status;

typedef enum { ADP_F64 = 0, ADP_F32 = 1 } adp_precision;

typedef enum {
    ADP_REG_HUBER_TV = 0,  /* phi(t) = t^2/(2 gamma) if |t| <= gamma else |t| - gamma/2  */
    ADP_REG_SQRT_TV = 1,   /* phi(t) = sqrt(t^2 + nu^2) - nu  (Sec. 4.2, smoothed TV)   */
    ADP_REG_QUAD = 2       /* phi(t) = t^2 / 2  (quadratic; closed-form checks)          */
} adp_reg;

typedef struct {
    int C, H, W, K;          /* channels, image size, odd kernel size K (1..63)          */
    double alpha;            /* lower-level weight of J                                   */
    double reg_param;        /* gamma (Huber) or nu (sqrt); ignored for ADP_REG_QUAD      */
    int reg;                 /* adp_reg                                                   */
    double beta;             /* Sobolev weight of the upper level                         */
    double sobolev_w0;       /* weight of ||b-a||^2 inside the H1 norm (1 full, 0 semi)  */
    int prec;                /* adp_precision                                             */
    double wait_timeout_s;   /* bound on each device-side wait; <= 0 selects 2 s          */
} adp_params;

typedef struct adp_problem adp_problem;

/* Creates a problem for data y (C x H x W) and the fixed kernel a of A
 * (C x K x K); both are copied into library-owned device memory, so the caller
 * may free them afterwards.  `stream` is a cudaStream_t (NULL = legacy default
 * stream).  Allocates the workspace (about 12 images) with cudaMalloc. */
adp_status adp_problem_create(const adp_params *params, const void *y, const void *a,
                              void *stream, adp_problem **out);
void adp_problem_destroy(adp_problem *p);

/* out = B x (Eq. 2.4, convolution with b).  x, out: C x H x W; b: C x K x K. */
adp_status adp_apply_B(adp_problem *p, const void *b, const void *x, void *out);
/* out = B^T z (the adjoint: correlation with b). */
adp_status adp_apply_Bt(adp_problem *p, const void *b, const void *z, void *out);

/* The same operators with BF16 operands and FP32 accumulation, on the tensor
 * cores (the BF16-input precision of the operator applications of Eq. 2.4):
 * x (or z) and b are rounded to BF16 (round to nearest even), every product
 * of two BF16 values is exact in FP32, and the K^2 products of an output are
 * summed in FP32 in tensor memory.  Only for ADP_F32 problems (float
 * pointers) with K <= 33; otherwise ADP_EINVAL.  The first call allocates the
 * operator's workspace (a BF16 copy of one image with periodic borders and
 * the kernel's Toeplitz bands, about C*(H+K)*(W+K)*2 + C*K*4096 bytes), which
 * the problem keeps until it is destroyed.  Each call runs three kernels on
 * the problem's stream (kernel bands, image conversion, correlation);
 * adp_last_kernel_ms reports the correlation alone and
 * adp_bf16_prep_ms_last the two preparation kernels. */
adp_status adp_apply_B_bf16(adp_problem *p, const void *b, const void *x, void *out);
adp_status adp_apply_Bt_bf16(adp_problem *p, const void *b, const void *z, void *out);
double adp_bf16_prep_ms_last(adp_problem *p);
/* CTAs of the tensor-core correlation's launch (0 before the first call). */
int adp_bf16_grid_size(adp_problem *p);

/* Operator path of the problem's later calls.  With enable = 1, every
 * application of B, B^T and A inside the library's calls (adp_apply_B/Bt,
 * the lower solve, the Hessian products of CG, the upper loss, the
 * kernel-gradient correlation, MAID) is evaluated through the convolution
 * theorem: with periodic boundaries B x is the circular convolution of x with
 * k(u, v) = b[u + r, v + r] (Eq. 2.4), so B x = F^-1(F(k) . F(x)),
 * B^T z = F^-1(conj(F(k)) . F(z)) and B^T B x = F^-1(|F(k)|^2 . F(x)), with
 * 2-D FFTs in FP32 (radix-2, twiddles rounded once from double); the
 * kernel-gradient correlation's K^2 lag sums are read off the inverse
 * transform of F(B v) conj(F(x)) + F(B x - y) conj(F(v)).  The cost no longer
 * grows with K^2.  Only for ADP_F32 problems whose H and W are powers of two
 * (2..8192) and whose rows and columns fit the kernel's shared memory;
 * otherwise ADP_EINVAL and the path is unchanged.  The first enable allocates
 * 32 bytes per value, C x H x W x 32 bytes in all (three complex images and two
 * real ones; kept until the problem is destroyed).
 * enable = 0 returns to the direct correlation; enable = 2 selects the FFT
 * path with the complex pipeline only (no real-to-complex pipeline, see
 * adp_fft_pipeline).  The FFT-path kernel runs 16 warps per CTA with the
 * problem's grid and all the shared memory a co-resident CTA may have;
 * ADP_EINVAL when that grid cannot be co-resident.  A batch (adp_batch_*) of
 * one problem follows the problem's path; batches of several problems use the
 * direct correlation. */
adp_status adp_set_fft(adp_problem *p, int enable);
int adp_fft_enabled(adp_problem *p);
/* Which pipeline carries the FFT path's lower-level solves: 0 the direct
 * correlation (FFT path off), 1 complex 2-D transforms of the whole image,
 * 2 the real-to-complex pipeline.  With the FFT path on and W >= 4, when its
 * staging fits in shared memory, the FISTA iteration of adp_lower_solve (and
 * of the solves inside adp_maid_step) runs as two grid phases: row transforms
 * of row pairs packed as one complex row, fused with the gradient, the
 * updates and the next iterate's forward transform; then the column
 * transforms of the half spectrum (columns 0 .. W/2) with the symbol
 * |F(k)|^2 of B^T B, less F(B^T y) (computed once per solve).  The CG of
 * adp_hypergrad (and of MAID) takes the same path for its Hessian products.
 * Its extra buffers (about C*H*W*14 bytes) are allocated by adp_set_fft. */
int adp_fft_pipeline(adp_problem *p);

/* out = grad_x h(x, b) = B^T(B x - y) + alpha grad J(x)   (Prop. 1, gradient);
 * *norm = ||out||_2 accumulated in FP64.  `out` may be NULL. */
adp_status adp_grad_lower(adp_problem *p, const void *b, const void *x, void *out, double *norm);

/* out = grad^2_x h(x, b) v = B^T B v + alpha D^T(phi''(D x) . D v)   (Prop. 1, Hessian). */
adp_status adp_hess_vec(adp_problem *p, const void *b, const void *x, const void *v, void *out);

/* Algorithm 1, step 1: FISTA on h(., b) from the warm start held in x,
 * stopped when ||grad_x h(y_k, b)|| <= eps (the test of Algorithm 1 with
 * mu := 1) or after max_iters updates; x receives y_k.  Step 1/L_c per channel
 * with L_c = ||b_c||_1^2 + 8 alpha sup phi''.  *iters = updates made,
 * *gradnorm = ||grad_x h|| at the returned point.  Returns ADP_ENOCONV when
 * the cap was reached (x still valid). */
adp_status adp_lower_solve(adp_problem *p, const void *b, void *x, double eps, int max_iters,
                           int *iters, double *gradnorm);

/* Upper-level loss ell = g(x) + r(b) and ||grad_x ell|| = ||grad g(x)||, the
 * terms of Eq. 3.4.  gradx (optional, may be NULL) receives grad g(x) =
 * 2 A^T (A x - y). */
adp_status adp_upper_loss(adp_problem *p, const void *b, const void *x, double *loss,
                          double *gradx_norm, void *gradx);

/* Algorithm 1, steps 2-3: conjugate gradients on grad^2_x h(x, b) q = rhs
 * from the start held in q (pass zeros for the paper's q_0 = 0), stopped at
 * ||residual|| <= delta or after max_iters iterations; then
 * z = -(grad^2_{xb} h(x, b))^T q + grad r(b).  With rhs == NULL the right-hand
 * side is grad g(x) (the hypergradient of Eq. 3.2); with an explicit rhs
 * (C x H x W, e.g. an upstream gradient) the grad r(b) term is left out.
 * q: C x H x W in/out; z: C x K x K out.  Returns ADP_ENOCONV at the cap. */
adp_status adp_hypergrad(adp_problem *p, const void *b, const void *x, const void *rhs,
                         double delta, int max_iters, void *q, void *z, int *cg_iters,
                         double *resnorm);

/* The kernel-gradient correlation of Algorithm 1, step 3, alone:
 * out[c,p,q] = sum_{i,j} x[c,i-p+r,j-q+r] (B v)[c,i,j] + v[c,i-p+r,j-q+r] (B x - y)[c,i,j]
 * = (grad^2_{xb} h(x, b))^T v.  out: C x K x K. */
adp_status adp_cross_t(adp_problem *p, const void *b, const void *x, const void *v, void *out);

/* State of Algorithm 2 carried between upper iterations, plus the report of
 * the last call.  Initialise with adp_maid_init (paper defaults, Sec. 4.1). */
typedef struct {
    double eps, delta, step;          /* eps_k, delta_k, alpha_k                         */
    double lambda;                    /* lambda of Eq. 3.4 (1e-4)                         */
    double rho_up, rho_down;          /* 1.1, 0.5                                         */
    double nu_up, nu_down;            /* 1.25, 0.5                                        */
    double L_gx;                      /* Lipschitz constant of grad g; set by adp_maid_init */
    double eps_stop;                  /* stop rule of Sec. 4.2: the upper iterations end once
                                         eps <= eps_stop (0 turns the rule off)            */
    int max_bt, max_rounds;           /* first inner-loop length (5), outer rounds (20)    */
    int ll_max_iters, cg_max_iters;   /* 300 (Sec. 4.1), 1000                             */
    int k;                            /* accepted upper iterations so far                  */
    /* report of the last adp_maid_step */
    int accepted, rounds, trials, ll_iters, cg_iters, ll_capped, cg_capped;
    int stopped;                      /* the stop rule fired (b, x unchanged)              */
    double loss, gradx_norm, znorm, psi;
} adp_maid_state;

/* Fills `s` with the paper's defaults, eps_stop = 0 (rule off) and
 * L_gx = 2 max_c ||a_c||_1^2. */
adp_status adp_maid_init(adp_problem *p, adp_maid_state *s);

/* One upper iteration of Algorithm 2 (MAID), entirely on the device in one
 * cooperative launch: InexactGradient(b_k, eps_k, delta_k), then backtracking
 * on psi <= 0 (Eq. 3.4) with lower-level re-solves warm-started from x~(b_k);
 * on success b_{k+1} = b_k - alpha_k z_k and eps, delta, alpha grow; after a
 * failed round eps and delta shrink and the gradient is recomputed.
 * b (C x K x K) and x (C x H x W, x~(b_k) in, x~(b_{k+1}) out) are in/out; q
 * (C x H x W) receives the last CG solution.  Returns ADP_ELSFAIL when all
 * rounds failed (b, x unchanged; s reports the shrunk eps, delta, step).  The
 * stop rule (eps <= eps_stop) is checked on entry and after every decrease of
 * eps; when it fires the call returns ADP_OK with s->stopped = 1,
 * s->accepted = 0 and b, x unchanged. */
adp_status adp_maid_step(adp_problem *p, adp_maid_state *s, void *b, void *x, void *q);

/* ---------------------------------------------------------------- batches
 * Many independent problems in one cooperative launch (uneven image sizes and
 * kernel sizes; one precision and device).  The grid is split into one group
 * of CTAs per problem; a group has its own barrier counter, reductions and
 * result record, and runs that problem's program exactly as a launch of its
 * own would (with fewer CTAs).  Group sizes start proportional to each
 * problem's convolution work (strips x K^2) and, after every
 * adp_batch_maid_step, are re-balanced from the measured time of each group
 * (half the old estimate, half the measurement) so that the groups finish
 * together; at most one group per co-resident CTA, and no group larger than
 * the problem's own launch.  There is no counterpart in the paper: this is the
 * batched form of adp_maid_step. */
typedef struct adp_batch adp_batch;

/* Groups n problems; they must outlive the batch.  Launches go to problem 0's
 * stream.  Allocates small device tables (cudaMalloc).  ADP_EINVAL for a mix
 * of precisions or devices, or more problems than co-resident CTAs. */
adp_status adp_batch_create(adp_problem *const *ps, int n, adp_batch **out);
void adp_batch_destroy(adp_batch *bt);

/* One upper iteration of Algorithm 2 on every problem of the batch in one
 * launch: st[i], b[i], x[i], q[i] are problem i's arguments of
 * adp_maid_step.  Returns ADP_OK when every problem accepted a step or has
 * stopped; otherwise the first failure (ADP_ELSFAIL when a problem exhausted
 * its backtracking rounds: its st[i] reports the shrunk eps, delta, step). */
adp_status adp_batch_maid_step(adp_batch *bt, adp_maid_state *st, void *const *b, void *const *x,
                               void *const *q);

/* A device-resident MAID run: max_steps batched upper iterations captured
 * once into a CUDA graph and replayed with no host round trip.  The MAID
 * state of every problem stays on the device between steps; a problem stops
 * for good at the stop rule (eps <= eps_stop) or when a step exhausts its
 * rounds, and its later steps return at once.  st[i] receives the final
 * eps, delta, step, k, the report of the last launch and `stopped`; totals
 * (optional, 4 values per problem) the run's FISTA + CG iterations,
 * convolution passes, upper iterations that ran, and accepted steps.  The
 * partition is the batch's current one. */
adp_status adp_batch_maid_run_graph(adp_batch *bt, adp_maid_state *st, void *const *b, void *const *x,
                                    void *const *q, int max_steps, long long *totals);

/* CTAs of problem i's group in the next launch; device time (ms) of the last
 * batched launch (adp_batch_maid_step) or graph (adp_batch_maid_run_graph). */
int adp_batch_group_size(adp_batch *bt, int i);
double adp_batch_last_kernel_ms(adp_batch *bt);

/* Launch shape of p's direct-path kernel (no counterpart in the paper: the
 * tile-shape knob of a launch-shape autotuner): grid CTAs of nw warps (even,
 * 2..8).  Strips of 32 x MR pixels are dealt to the grid's warps, so the
 * shape decides how evenly the strips of a pass spread, and how many warps
 * share an SM.  ADP_EINVAL when the warps' stages do not fit in shared memory
 * or the grid cannot be co-resident; the reduction slots grow (cudaMalloc) when
 * the new shape needs more.  Set it before adp_set_fft and before creating a
 * batch with p (both take the problem's shape then).  The problem's initial
 * shape is one CTA per SM of the most warps that fit, or enough CTAs for a
 * strip per warp. */
adp_status adp_set_launch(adp_problem *p, int grid, int nw);

/* Diagnostics of the last call on p: number of full-image convolution passes
 * it executed (each is 2 K^2 C H W flops; the kernel-gradient correlation
 * counts as two), and the number of CTAs of its cooperative launch. */
long long adp_conv_passes_last(adp_problem *p);
int adp_grid_size(adp_problem *p);
/* Warps per CTA of the problem's launches (chosen from the shared memory a
 * warp's halo tiles need for this kernel size). */
int adp_warps_per_cta(adp_problem *p);
/* Device time in ms of the last call's cooperative kernel, measured with CUDA
 * events recorded on the problem's stream around the launch. */
double adp_last_kernel_ms(adp_problem *p);

/* Lower-level solve that allocates nothing.  There is no counterpart in the
 * paper: this is an engineering variant of adp_lower_solve for callers that
 * cannot allocate device memory when they need a solve -- cudaMalloc/cudaFree
 * synchronise the device (unacceptable inside a latency-critical or real-time
 * loop), and callers that give all device memory to their own pool or run
 * under a memory budget fixed at start-up must not have a library allocate.
 *
 * Same computation as adp_lower_solve (FISTA on h(., b) from the warm start in
 * x, stopped at ||grad_x h(y_k, b)|| <= eps or after max_iters updates; x
 * receives y_k; ADP_ENOCONV at the cap), but without an adp_problem: y
 * (C x H x W), b (C x K x K) and x are the caller's device pointers, `stream`
 * a cudaStream_t, and the workspace is one fixed array in the library's
 * device memory, ADP_NOALLOC_SCRATCH_BYTES in size, which every GPU that
 * loads the library holds until the process exits.  The solve keeps seven
 * images in the padded layout of the library (periodic ghost borders of
 * Gy = max(r, 1) rows and Gx = max(r rounded up to 4, 4) columns, rows padded
 * to a multiple of 4 elements; r = (K-1)/2), each limited to
 * C*(H+2Gy)*round_up(W+2Gx, 4)*element size <= ADP_NOALLOC_MAX_IMAGE_BYTES
 * (e.g. 3 x 512 x 512 in FP32 with any K up to 63), and the kernel weights to
 * 4*C*K*round_up(K, 16 in FP32 or 8 in FP64)*element size <=
 * ADP_NOALLOC_WEIGHT_BYTES; larger problems are rejected with ADP_EINVAL.
 * The first call on a device looks up the array's device address and sets
 * kernel attributes for that device (once per device, with it current); make
 * that first call before any stream capture.  Every call waits for its
 * stream to finish the solve and reads the iteration count and gradient norm
 * back to the host before it returns.  The device used is the current one:
 * the pointers and the stream must belong to it.  All calls share the array and
 * it keeps the last call's contents (each call clears what must start at
 * zero), so calls whose GPU work overlaps -- on different streams, or from
 * different threads -- race and must be serialised by the caller.  Calls no
 * cudaMalloc, cudaFree or other allocating routine. */
#define ADP_NOALLOC_MAX_IMAGE_BYTES 4194304
#define ADP_NOALLOC_WEIGHT_BYTES 1048576
#define ADP_NOALLOC_SCRATCH_BYTES (512 + 8 * 512 * 8 + ADP_NOALLOC_WEIGHT_BYTES + 7 * ADP_NOALLOC_MAX_IMAGE_BYTES)
adp_status adp_lower_solve_noalloc(const adp_params *params, const void *y, const void *b, void *x, double eps,
                                   int max_iters, void *stream, int *iters, double *gradnorm);

/* ------------------------------------------------------------------------
 * 1D elastic-net variant (Sec. 4.1).  The operator is a full n x n matrix B
 * (the kernel b(t, tau) of Eq. 2.4 sampled on the signal's grid), learned with
 * beta = 0, so the upper level is l(B) = ||A x(B) - y||^2 (Eq. 2.5a) and the
 * lower level is h(x; B) = 1/2 ||B x - y||^2 + a1 ||x||_1 + a2 ||x||_2^2,
 * solved by proximal gradient with step lam (Sec. 4.1).  The accuracy of a
 * lower-level iterate is the norm of the proximal-gradient mapping
 * G(x) = (x - prox(x - lam B^T (B x - y))) / lam; the hypergradient solves the
 * Hessian system on the support S = {i : x_i != 0} of x by CG and is the
 * rank-two matrix z = -((B x - y) q^T + (B q) x^T) (Algorithm 1).
 *
 * Every call runs on one thread-block cluster of 8 CTAs: for each operator it
 * solves with, each CTA forms 1/8 of the rows of B^T B and B^T y in shared
 * memory, and the CTAs exchange vector slices through distributed shared
 * memory.  FP32 matrices and
 * vectors; dot products, norms and the line-search test in FP64.  Matrices
 * are row-major n x n FP32 device arrays, vectors n FP32 device arrays, all
 * owned by the caller; calls are ordered on the problem's stream and wait for
 * it before returning their scalar outputs.  Errors: ADP_EINVAL for bad
 * arguments (n not a multiple of 32 or above ADP_EN1D_MAX_N, null pointers,
 * a1, a2 < 0, lam <= 0), ADP_ENOMEM / ADP_ECUDA as for the 2D problem. */
#define ADP_EN1D_MAX_N 384
typedef struct {
    int n;              /* signal length, a multiple of 32, 32 .. ADP_EN1D_MAX_N */
    double a1, a2;      /* elastic net a1 ||x||_1 + a2 ||x||_2^2 (1.2e-3, 4e-3)  */
    double lam;         /* proximal-gradient step (0.1)                         */
} adp_en1d_params;
typedef struct adp_en1d adp_en1d;

/* A: the forward matrix (n x n), y: the data (n); both device pointers, read
 * by every later call (the caller keeps them alive).  stream: a cudaStream_t
 * or NULL. */
adp_status adp_en1d_create(const adp_en1d_params *params, const float *A, const float *y, void *stream,
                           adp_en1d **out);
void adp_en1d_destroy(adp_en1d *p);

/* Proximal gradient from x (in: warm start, out: the result) for the
 * operator B: returns the first iterate with ||G|| <= eps, or the iterate
 * after max_iters updates; iters = updates made, gmap_norm = its ||G||. */
adp_status adp_en1d_lower_solve(adp_en1d *p, const float *B, float *x, double eps, int max_iters, int *iters,
                                double *gmap_norm);

/* l = ||A x - y||^2 and ||grad g(x)|| = ||2 A^T (A x - y)||. */
adp_status adp_en1d_upper_loss(adp_en1d *p, const float *x, double *loss, double *gradx_norm);

/* Algorithm 1, steps 2-3, on the support of x: CG from q = 0 on
 * (B^T B + 2 a2 I)_SS q_S = grad g(x)_S until ||r|| <= delta or max_iters
 * iterations, q = 0 off S; then z = -((B x - y) q^T + (B q) x^T).  q: n,
 * z: n x n, both written. */
adp_status adp_en1d_hypergrad(adp_en1d *p, const float *B, const float *x, double delta, int max_iters, float *q,
                              float *z, int *cg_iters, double *resnorm);

/* Algorithm 2 with Sec. 4.1's constants: adp_en1d_maid_init fills s (eps =
 * delta = 1e-2, alpha = 0.1, the 2D problem's line-search constants, 300
 * lower-level iterations, L_gx = 2 ||A||_1 ||A||_inf).  adp_en1d_maid_step
 * runs one upper iteration in one cluster launch and updates B and x in
 * place on acceptance (the same report fields as adp_maid_step; a step that
 * exhausts its rounds or meets the stop rule leaves B and x as they were).
 * adp_en1d_maid_run runs up to max_steps upper iterations in one launch,
 * ending early when the stop rule fires or a step exhausts its rounds;
 * steps = upper iterations run. */
adp_status adp_en1d_maid_init(adp_en1d *p, adp_maid_state *s);
adp_status adp_en1d_maid_step(adp_en1d *p, adp_maid_state *s, float *B, float *x);
adp_status adp_en1d_maid_run(adp_en1d *p, adp_maid_state *s, float *B, float *x, int max_steps, int *steps);

/* Diagnostic of the failure path (no counterpart in the paper): one launch
 * of p's kernel in which CTA 0 never arrives at a grid barrier, so the bounded
 * wait of every other CTA runs out after the problem's wait_timeout_s.  The
 * expected result is ADP_ETIMEOUT, returned without a fault, with p and the
 * CUDA context still usable.  ADP_EINVAL when p's launch has a single CTA. */
adp_status adp_selftest_wait_timeout(adp_problem *p);

/* Tracing (diagnostics).  With cap > 0, later calls on p record, for the first
 * cap grid barriers of each launch, the device global timer (ns) when CTA 0
 * arrived at and left the barrier; cap = 0 turns tracing off.  Allocates (and
 * frees) a device buffer of 2 * cap values with cudaMalloc/cudaFree.
 * adp_trace_read copies the (arrive, leave) pairs of the last call to host
 * memory (at most cap pairs) and returns how many pairs it wrote, or -1. */
adp_status adp_trace_enable(adp_problem *p, int cap);
int adp_trace_read(adp_problem *p, long long *host_out, int cap);

/* Thread-local message for the last failing call on this thread. */
const char *adp_last_error(void);
const char *adp_status_string(adp_status s);

#ifdef __cplusplus
}
#endif

#endif /* ADP_H */
