/*
 * libph -- online stage of parametric H- and H^2-matrices on one GB300 (sm_103a).
 *
 * Method: Khan, Chen, Rao, Saibaba, "Parametric Hierarchical Matrix
 * Approximations to Kernel Matrices".  The problem statement (§1): for points
 * X = (x_i) in a box B of R^d and a parametric kernel kappa(x, y; theta) with
 * theta in a box B_theta of R^{d_theta}, approximate K(X, X; theta) once
 * (offline) so that for any theta the hierarchical matrix K_hat(theta) can be
 * instantiated without new kernel evaluations and applied to vectors (online).
 *
 * Conventions shared by every call:
 *   - Every call returns a ph_status; no C++ exception crosses this boundary.
 *     On failure, ph_last_error(handle) (or ph_last_error(NULL) when no handle
 *     exists) returns a one-line description.
 *   - Device pointers are plain CUDA global-memory addresses on the handle's
 *     device; host pointers are ordinary process memory.
 *   - Matrices are column-major: element (i, j) of an n x m matrix with
 *     leading dimension ld is at [i + j * ld], ld >= n.
 *   - Streams are passed as `void*` holding a cudaStream_t (NULL = default
 *     stream).  ph_instantiate and ph_matvec are stream-ordered and
 *     asynchronous; one handle must not be used on two streams at once.
 *   - The scalar type of X and Y is double for PH_FP64 handles and float for
 *     PH_FP32 handles.
 */
#ifndef PH_H
#define PH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ph_handle ph_handle;

typedef enum {
    PH_OK = 0,
    PH_ERR_INVALID_ARG = 1,       /* bad pointer, size, option or point outside the root box */
    PH_ERR_THETA_OUT_OF_BOX = 2,  /* theta outside B_theta: the interpolant is defined on B_theta only */
    PH_ERR_NOT_INSTANTIATED = 3,  /* ph_matvec before any successful ph_instantiate */
    PH_ERR_OOM = 4,               /* host or device allocation failed */
    PH_ERR_CUDA = 5,              /* a CUDA, cuBLAS or cuSOLVER call failed (no device, launch error ...) */
    PH_ERR_NONFINITE = 6,         /* non-finite theta, or non-finite X when check_finite is set */
    PH_ERR_TIMEOUT = 7,           /* a bounded device-side wait ran out: the result of the call it
                                     ran out in is invalid.  Reported by that call when it
                                     synchronises (check_finite set), else by ph_check, or by the
                                     first ph_instantiate / ph_matvec* call on the handle made
                                     after the stream passed that call, which then does no work
                                     (call it again to proceed) */
    PH_ERR_IO = 8,                /* ph_save / ph_load file error or bad file */
    PH_ERR_UNSUPPORTED = 9        /* option combination not implemented */
} ph_status;

/* Kernel functions kappa(x, y; theta), r = |x - y|_2.  The first three are the
 * workloads' kernels; SE, E and MQ are the paper's (§6 kernel table);
 * POLY / POLYXY are exact-interpolation test kernels. */
typedef enum {
    PH_KERNEL_GAUSS = 0,        /* exp(-r^2 / (2 l^2)),                     theta = (l)        */
    PH_KERNEL_MATERN32 = 1,     /* (1 + sqrt(3) r/l) exp(-sqrt(3) r/l),     theta = (l)        */
    PH_KERNEL_MATERN52 = 2,     /* (1 + sqrt(5) r/l + 5 r^2/(3 l^2)) exp(-sqrt(5) r/l)          */
    PH_KERNEL_ANISO_GAUSS = 3,  /* exp(-sum_k (x_k - y_k)^2 / (2 l_k^2)),   theta = (l_1..l_d) */
    PH_KERNEL_SE = 4,           /* exp(-(r/l)^2)                                                */
    PH_KERNEL_EXPONENTIAL = 5,  /* exp(-r/l)                                                    */
    PH_KERNEL_MULTIQUADRIC = 6, /* (1 + (r/l)^2)^(1/2)                                          */
    PH_KERNEL_POLY = 7,         /* 1 + theta r^2 + theta^2 r^4                                  */
    PH_KERNEL_POLYXY = 8,       /* (1 + x.y)^2 (1 + theta); not translation-invariant           */
    PH_KERNEL_POLY2 = 9         /* 1 + theta_1 r^2 + theta_2^2 r^4,         theta = (th_1, th_2) */
} ph_kernel;

typedef enum { PH_FMT_H2 = 0, PH_FMT_H = 1 } ph_format;       /* Definitions of §4.1 */
typedef enum { PH_FP64 = 0, PH_FP32 = 1 } ph_precision;       /* stored cores and online arithmetic */

/* Options of the offline stage (Algs. "Offline Stage: Parametric H-matrix" and
 * "... H^2-matrix", §4.4).  Fixed-size arrays keep the struct plain. */
typedef struct {
    int d;                 /* spatial dimension, 1..3 */
    int dtheta;            /* parameter dimension 1..3; the tensor grid has prod_i (degree_i + 1) <= 1024 points,
                              and with d_theta > 1 the far ranks around the parameter cores must be <= 64 */
    double theta_lo[3];    /* parameter box B_theta = prod [theta_lo_i, theta_hi_i] */
    double theta_hi[3];
    int degree[3];         /* Chebyshev degree in theta_i; p_theta_i = degree_i + 1 nodes (§2.2) */
    int p_s;               /* spatial Chebyshev nodes per dimension (§2.2), 1..16 */
    int l_max;             /* depth of the uniform 2^d-ary cluster tree (§3.2), 0..10 */
    double eta;            /* admissibility parameter (§3.4) */
    double tol;            /* TT-SVD tolerance eps for the far field */
    double near_tol;       /* TT-SVD tolerance for the near field; < 0 means tol */
    int rank_cap;          /* cap on every far-field TT rank; 0 = no cap */
    ph_format fmt;
    ph_precision prec;
    int dedup;             /* 1: compress one far tensor per (level, offset) class (§5.2);
                              forced off for kernels that are not translation-invariant */
    int check_finite;      /* 1: ph_matvec checks X for non-finite entries (synchronises) */
    int device;            /* CUDA device ordinal */
    int coupling;          /* H^2 coupling stage: 0 = explicit factors L_k, R_k per translation class
                              applied as two matrix products (the alternative §4.5 mentions),
                              1 = the TT chain of Alg. "Modified H^2-Matrix MVM"; mode 0 needs
                              r_d, r_{d+d_theta} <= 64 and falls back to 1 otherwise */
    int near_unshared;     /* 0 (default): store each unordered near pair {s, t} once and apply the
                              mirror block as D_ts(theta) = D_st(theta)^T.  Every kernel here is
                              symmetric, so A_ts is a row permutation of A_st and TT-SVD gives the
                              same cores up to that permutation (§4.3): the sharing is exact and
                              halves the near-field stream.  1: compress and store both blocks. */
    int near_degree[3];    /* Chebyshev degree in theta_i of the near-field tensor grid (§4.3); 0 = degree[i].
                              The near and far grids are independent: each field interpolates on its own
                              nodes (the near field often needs fewer, e.g. 5 per dimension for
                              d_theta = 3).  ph_matvec_batched then applies one theta at a time. */
    int compressor;        /* far-field tensors: 0 (default) TT-SVD of the formed tensor on the GPU (QR +
                              SVD per cut, FP64); 1 greedy TT-cross + TT-rounding on the host (§2.1, the
                              paper's compressor), which evaluates only the entries it needs.  The
                              near field always uses TT-SVD. */
} ph_build_opts;

/* Sizes and counts of a built handle; all byte counts are of stored data. */
typedef struct {
    long n;                  /* points */
    int d, dtheta, p_s, p_theta[3];
    int prec, fmt;
    int n_nodes, n_leaves, tree_depth;
    long n_near, n_far, n_far_keys;   /* near blocks, far blocks, compressed far tensors */
    long near_entries;       /* sum over near blocks of n_s * n_t */
    long near_rank_sum;      /* sum over near blocks of r_{b,1} */
    int near_rank_max, far_rank_max;
    double far_rank_mean;    /* mean over far blocks of max(r_{b,d}, r_{b,d+dtheta}) (paper's "Rank", §6) */
    long near_bytes;         /* stored near-field cores G_{b,1} (the online stream) */
    long near_theta_bytes;   /* stored near-field theta cores */
    long far_bytes;          /* far-field cores (all keys), plus S_b / T_b for the H format */
    long basis_bytes;        /* leaf factor matrices U_{s,k} and transfer factors */
    double alg_bytes_per_call;   /* bytes one ph_instantiate + ph_matvec with m = 1 must move
                                    (excluding X / Y); add 2 * n * m * scalar for X and Y */
    double flops_per_rhs;    /* online flops per right-hand side (instantiate excluded) */
    double offline_seconds;  /* wall time of ph_offline_build */
    double coupling_a_flops_per_rhs;  /* explicit coupling phase 1 (H_k R_k^T xhat), or the whole TT chain */
    double coupling_b_flops_per_rhs;  /* explicit coupling phase 2 (sum L_k z_b); 0 for the TT chain */
    int tensor_core_phase1;  /* 1 when calls with 8 < m <= 16 run phase 1 of the explicit coupling
                                on the tensor cores (see ph_set_tensor_cores), else 0 */
    int kernel_variants;     /* kernels the last ph_matvec on this handle launched: bit 0 the
                                bulk-copy near field, bit 1 the bulk-copy phase 2 of the
                                coupling, bit 2 the tensor-core phase 1 (0 before any call) */
    long far_core_elems;     /* sum over translation classes of r_d r_{d+d_theta}: the instantiated
                                far-field cores H_k(theta) (and the surrogate's outputs) */
    int p_theta_near[3];     /* nodes per parameter dimension of the near-field grid */
} ph_info;

/* Build the parametric matrix (offline stage).
 *   points : host, n x d, row-major doubles (point i at points[i*d .. i*d+d-1]),
 *            read only during the call; every point must lie in [0,1]^d (§6).
 *   out    : receives a new handle owning all host and device data.
 * The tree is the uniform tree of §3.2 (depth l_max), the block tree that of
 * §3.4; near blocks are compressed by TT-SVD of A_b (§4.3), far blocks by
 * TT-SVD of M_b (§4.2, App. A.4).  Runs on the GPU (FP64). */
ph_status ph_offline_build(const double* points, long n, ph_kernel kernel,
                           const ph_build_opts* opts, ph_handle** out);

/* Online stage (Alg. "Online Stage", §4.4): evaluate the parametric vectors
 * v_i(theta_i) (App. A.4) in FP64, the near-field weights prod_i G_{b,i+1} x_2 v_i
 * (§4.3) and the far-field core matrices H_b(theta) (Alg. PTTK online, App. A.4).
 *   theta : host, d_theta doubles; must lie in B_theta.
 * Stream-ordered; theta is copied before the call returns. */
ph_status ph_instantiate(ph_handle* h, const double* theta, void* stream);

/* The theta-derivative of the instantiated matrix: as ph_instantiate, with the parametric
 * vector of dimension `dim` replaced by the derivatives of its Lagrange polynomials,
 * [v_dim']_k = d ell_k / d theta_dim (the other dimensions keep v_i).  Every stored
 * quantity enters linearly in each v_i (§4.3 near weights, App. A.4 H_b), so the handle
 * then holds dK_hat(theta) / dtheta_dim and ph_matvec applies it.  The derivative weights
 * are FP64, by the barycentric derivative (Berrut & Trefethen 2004, §9; the
 * differentiation-matrix form when theta is a node).  Not in the paper: it serves gradients
 * of GP hyperparameter objectives.  Errors: as ph_instantiate, plus PH_ERR_INVALID_ARG when
 * dim is not in [0, d_theta).  Stream-ordered; theta is copied before the call returns. */
ph_status ph_instantiate_derivative(ph_handle* h, const double* theta, int dim, void* stream);

/* Y = K_hat(theta) X for the last instantiated theta (§4.5: the H-matrix MVM with
 * S_b H_b T_b^T far blocks, or Alg. "Modified H^2-Matrix MVM").
 *   X : device, n x m column-major, leading dimension ldx >= n, original point order.
 *   Y : device, n x m column-major, leading dimension ldy >= n; overwritten.
 *   m : number of right-hand sides, 1..1024.
 * X and Y must not overlap.  Stream-ordered and asynchronous. */
ph_status ph_matvec(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy,
                    void* stream);

/* X = K_hat(theta)^T Y for the last instantiated theta (or the transpose of its theta-derivative
 * after ph_instantiate_derivative): the adjoint of ph_matvec, the gradient of a scalar function
 * of Y = K_hat X with respect to X.  Not in the paper (it serves gradients of GP objectives); every
 * block enters transposed: near blocks D_b(theta)^T (§4.3), far blocks T_b H_b^T S_b^T (H format,
 * §4.5) or C_b^T = R_b H_b^T L_b^T between the sweeps (H^2, §4.2, Alg. FastForward / FastBackward
 * on Y).  The first call builds the transposed far structure (the far blocks regrouped by source,
 * the factors of each class exchanged) and keeps it; later ph_instantiate calls also write H_k^T.
 *   Y : device, n x m column-major, leading dimension ldy >= n, original point order.
 *   X : device, n x m column-major, leading dimension ldx >= n; overwritten.
 * Errors: as ph_matvec, plus PH_ERR_UNSUPPORTED for an H^2 handle with the TT-chain coupling
 * (coupling = 1).  Stream-ordered and asynchronous. */
ph_status ph_matvec_transpose(ph_handle* h, const void* Y, long ldy, int m, void* X, long ldx, void* stream);

/* Many theta, one block of right-hand sides (d_theta = 1): Y_t = K_hat(theta_t) X for
 * t < n_theta, or dK_hat/dtheta(theta_t) X with deriv = 0 (deriv = -1: the matrix itself).
 * K_hat(theta) is linear in the parametric vector (§4.3 weights, App. A.4 H_b), so
 * K_hat(theta) X = sum_q ell_q(theta) K_hat(eta_q) X exactly over the p_theta Chebyshev nodes
 * eta_q.  With n_theta >= p_theta the call forms the p_theta products K_hat(eta_q) X once and
 * combines them per theta in one kernel (the weights in FP64, by the barycentric formula);
 * with fewer theta, and always for the derivative of an FP32 handle (whose node combination
 * would amplify FP32 rounding by the size of the derivative weights), it instantiates and
 * applies once per theta.  Not in the paper.
 *   thetas   : host, n_theta doubles, each in B_theta (1 <= n_theta <= 2,097,120).
 *   X        : device, n x m, column-major, leading dimension ldx >= n, original order.
 *   Y        : device, n_theta blocks n x m, block t at Y + t * stride_y (elements), leading
 *              dimension ldy >= n, stride_y >= ldy * m; overwritten.
 * Leaves the handle instantiated at an unspecified theta: call ph_instantiate before the
 * next ph_matvec.  Allocates p_theta * n * m scalars of workspace on first use (kept by the
 * handle).  Errors: PH_ERR_INVALID_ARG (sizes, deriv), PH_ERR_THETA_OUT_OF_BOX,
 * PH_ERR_NONFINITE (theta), PH_ERR_UNSUPPORTED (d_theta != 1), PH_ERR_OOM, PH_ERR_CUDA.
 * Stream-ordered; thetas are copied before the call returns. */
ph_status ph_matvec_batched(ph_handle* h, const double* thetas, int n_theta, const void* X, long ldx, int m,
                            void* Y, long ldy, long stride_y, int deriv, void* stream);

/* ph_matvec on HOST buffers: copies X to the device, applies K_hat(theta),
 * copies Y back and synchronises the stream before returning.  X and Y are
 * host pointers with the same layout as in ph_matvec (pinned memory makes the
 * copies asynchronous DMA). */
ph_status ph_matvec_host(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy,
                         void* stream);

/* ph_matvec for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a service of the library.  ph_matvec allocates its per-call
 * workspace with cudaMalloc the first time it meets a problem size, and cudaMalloc
 * may synchronise the device and can fail when memory is tight.  Some callers cannot
 * allow that when they apply the matrix: processes held to a fixed device-memory
 * budget that is fully committed after set-up, host applications that own every
 * device allocation through their own allocator, and latency-bound loops that must
 * not stall on an allocation.  This variant allocates nothing and calls no allocating
 * library routine (no cudaMalloc, no cudaFree, nothing from PyTorch).  Its workspace
 * lives in one file-scope device array of 16 MiB that every GPU loading the library
 * holds until the process exits.
 *   Arguments, layout, result and errors are those of ph_matvec; with check_finite set
 *     the call reads a flag back and synchronises the stream, as ph_matvec does.
 *   Sizes: the workspace needed is about 4 (float) or 8 (double) bytes times
 *     m_pad * (n + near work items * largest leaf + 2 * tree nodes * p_s^d
 *     + far blocks * largest r_d) (H^2) or m_pad * (n + items * largest leaf +
 *     far levels * n) (H), m_pad =
 *     m rounded up to 1, 2, 4, 8 or a multiple of 16; above 16 MiB the call
 *     returns PH_ERR_INVALID_ARG with the needed size in ph_last_error and
 *     computes nothing.
 *   Set-up: the first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   Sharing: every call uses the same array, which keeps the last call's
 *     contents (the call clears what must start at zero).  Calls whose work
 *     overlaps on the GPU, from any handle or stream, race on the array. */
ph_status ph_matvec_noalloc(ph_handle* h, const void* X, long ldx, int m, void* Y, long ldy,
                            void* stream);

/* Waits for the handle's work on `stream` (and on its internal far-field stream) and reports
 * PH_ERR_TIMEOUT if a bounded device-side wait of an earlier call ran out since the last
 * report (that call's result is invalid), else PH_OK; PH_ERR_CUDA if the stream reports an
 * error.  Synchronous.  Not in the paper: a status query of the library. */
ph_status ph_check(ph_handle* h, void* stream);

/* Test hook (the paper has no counterpart): runs, on `stream`, one CTA that waits on an mbarrier
 * nothing arrives on, with the bounded wait of the production kernels (about one second), and
 * counts the expiry in the handle's device flag exactly as a production kernel whose wait ran
 * out does.  The call itself returns PH_OK (asynchronous).  ph_check on the handle then reports
 * PH_ERR_TIMEOUT once; so does the first ph_instantiate / ph_matvec* call made after the stream
 * has passed the wait (after a synchronisation).  No kernel is faulted or hung. */
ph_status ph_selftest_timeout(ph_handle* h, void* stream);

/* Test hook (the paper has no counterpart): after `after` more successful device allocations
 * of the library in this process, every further one fails as if cudaMalloc had failed, so
 * that the caller sees PH_ERR_OOM; after < 0 switches the injection off.  A handle whose
 * allocation failed in ph_matvec stays valid (destroy it, or switch the injection off and
 * call again).  Affects every handle of the process; always returns PH_OK. */
ph_status ph_inject_alloc_failure(long after);

/* ------------------------------------------------------------------------------------------
 * Learned surrogate of the far-field cores.  The paper lists other parametric approximations as
 * future work (§7); this learned one is an extension, not the paper's method.  In the H^2 format with
 * the explicit coupling (coupling = 0) the only theta-dependent far-field quantity is the core
 * H_k(theta) of each translation class (App. A.4); the spatial factors L_k, R_k stay fixed.  A
 * perceptron theta -> (H_k(theta))_k replaces the polynomial contraction of the stored theta
 * cores when its validation error passes the acceptance test; otherwise the polynomial path stays.
 * None of these calls changes the polynomial data.  The network is not written by ph_save.
 * ------------------------------------------------------------------------------------------ */

/* The exact far-field cores in the gauge of the stored spatial factors, for n_theta parameters:
 *   H*_k(theta) = (L_k^T L_k)^{-1} L_k^T W_k(theta) R_k (R_k^T R_k)^{-1},
 * the least-squares solution of L_k H R_k^T = W_k(theta), W_k(theta) the coupling matrix of §3.6.2
 * (the kernel on the Chebyshev grids of the class's representative boxes) at theta.  These are the
 * surrogate's training targets.
 *   thetas : host, n_theta x d_theta (row-major), each inside the box (PH_ERR_THETA_OUT_OF_BOX).
 *   out    : device, n_theta x ph_info.far_core_elems scalars of the handle's precision; core k of
 *            theta t at out[t * far_core_elems + (offset of class k)], column-major r_d x r_{d+d_theta}
 *            (the layout ph_instantiate_cores reads).
 * H^2 with coupling = 0 only (else PH_ERR_UNSUPPORTED).  Asynchronous on `stream` after a
 * synchronous first-call set-up (the factors' Gram matrices, on the host in FP64). */
ph_status ph_far_project(ph_handle* h, const double* thetas, int n_theta, void* out, void* stream);

/* Instantiate at theta (as ph_instantiate for the near field) with the far-field cores copied from
 * `cores` (device, far_core_elems scalars in the layout of ph_far_project) instead of the
 * polynomial contraction.  Asynchronous. */
ph_status ph_instantiate_cores(ph_handle* h, const double* theta, const void* cores, void* stream);

/* Training options of the surrogate (zero fields take the default in brackets). */
typedef struct {
    int hidden;              /* width of both hidden layers [256] */
    int steps;               /* Adam steps [2000] */
    int batch;               /* samples per step [256] */
    double lr;               /* Adam learning rate, decayed by a cosine to lr / 100 [1e-3] */
    double accept_tol;       /* acceptance on the RMS validation error (ph_surrogate_report): > 0 accept
                                when the network's is at most this; 0 [default] accept when it is at
                                most the polynomial path's */
    unsigned long long seed; /* initial weights ~ N(0, 1 / fan_in) from this seed, and the batch order */
} ph_surrogate_opts;

/* What ph_surrogate_train measured on the validation thetas t.  Errors are taken on the coupling
 * matrices, E_t^2 = sum_k ||L_k (H_k - H*_k) R_k^T||_F^2 at t (computed in orthonormal bases of the
 * stored factors, where it is the Frobenius norm of the transformed core), with
 * S = sqrt(mean_t sum_k ||L_k H*_k R_k^T||_F^2) their RMS size:
 *   rms = sqrt(sum_t E_t^2 / sum_t sum_k ||L_k H*_k R_k^T||^2),   max = max_t E_t / S.
 * (Per-theta relative errors would be dominated by the thetas where the far field is negligible,
 * e.g. the shortest length scales; errors of H itself would weigh directions that the factors
 * scale down.) */
typedef struct {
    long params;             /* weights and biases of the network */
    long out_dim;            /* network outputs (= far_core_elems) */
    double loss_first, loss_last;  /* training loss of the first and the last step (scaled targets) */
    double val_err_net_rms, val_err_net_max;     /* the network's cores */
    double val_err_poly_rms, val_err_poly_max;   /* the polynomial path's cores */
    double targets_seconds, train_seconds;       /* wall time: targets (ph_far_project), training */
    int accepted;            /* 1: ph_surrogate_use may switch the network on */
} ph_surrogate_report;

/* Train the surrogate on the GPU (forward, backward and Adam kernels of this library; BF16 weight
 * copies in the matrix products with FP32 accumulation, FP32 master weights):
 *   u = 2 (theta - lo) / (hi - lo) - 1,  h1 = gelu(W1 u + b1),  h2 = gelu(W2 h1 + b2),
 *   y = W3 h2 + b3,  K_k(theta) = s_k y_k,  H_k = A_{L,k}^{-1} K_k A_{R,k}^{-T},
 * gelu(x) = x Phi(x) (exact), A the upper Cholesky factors of L_k^T L_k and R_k^T R_k (so that K_k is
 * the core in orthonormal bases of the factors' column spaces), s_k the RMS of class k's training
 * targets.  Loss: mean squared error of y against the targets K*_k / s_k, K* = A_L H* A_R^T.  thetas_train / thetas_val: host, n x d_theta, inside the box
 * (the caller draws them).  The acceptance test compares the network's validation error with
 * opts->accept_tol or with the polynomial cores' (see ph_surrogate_opts).  rep may be NULL.
 * A later call replaces the network.  Synchronous. */
ph_status ph_surrogate_train(ph_handle* h, const double* thetas_train, int n_train, const double* thetas_val,
                             int n_val, const ph_surrogate_opts* opts, ph_surrogate_report* rep, void* stream);

/* enable = 1: ph_instantiate takes the far-field cores from the trained network (one forward pass
 * per theta); PH_ERR_UNSUPPORTED if no network was accepted (the polynomial path stays).  enable = 0
 * goes back to the polynomial path.  ph_instantiate_derivative and ph_matvec_batched's node
 * combination always use the polynomial path. */
ph_status ph_surrogate_use(ph_handle* h, int enable);

/* Test hook for the network kernels alone: one forward pass, loss and backward pass of a
 * perceptron n_in -> hidden -> hidden -> n_out on `batch` inputs, on the current device.
 *   params  : host FP32 [W1 (hidden x n_in) b1 W2 (hidden x hidden) b2 W3 (n_out x hidden) b3],
 *             row-major; the weights are used as BF16 (rounded to nearest even), biases as FP32
 *   U, T    : host, batch x n_in inputs (already in [-1, 1]) and batch x n_out targets
 *   Y       : host, receives batch x n_out outputs
 *   grads   : host, receives the gradient of the loss sum (Y - T)^2 / (2 batch n_out) in the layout
 *             of params (with respect to the weights as used)
 *   loss    : receives the loss. */
ph_status ph_mlp_check(int n_in, int hidden, int n_out, const float* params, int batch, const float* U,
                       const float* T, float* Y, float* grads, double* loss);

/* Test hook of the TT-cross compressor (no GPU involved): greedy TT-cross and TT-rounding (§2.1)
 * of a dense host tensor of q dimensions (Fortran order, dims[0] fastest) with tolerance eps and
 * rank cap (0: none).  Writes the ranks r_0..r_q (q + 1 ints), the reconstructed tensor (same
 * size and order as tensor) and the number of distinct entries the cross evaluated.  The offline
 * build uses the same routine on the far-field tensors when compressor = 1. */
ph_status ph_tt_cross_check(int q, const int* dims, const double* tensor, double eps, int cap, int* ranks,
                            double* approx, long* evals);

/* Test hook (no GPU): the offline build's TT-cross of one far-field tensor M_b (App. A.4): modes
 * (i_1..i_d, theta_1..theta_dtheta, j_1..j_d), entries kappa(x_i, y_j; theta) on the Chebyshev grids
 * of the target box [s_lo, s_hi], the source box [t_lo, t_hi] (p_s nodes per dimension) and the
 * parameter box (degree[k] + 1 nodes); writes the ranks (2d + dtheta + 1 ints) and the reconstructed
 * tensor (Fortran order, p_s^(2d) prod(degree + 1) doubles). */
ph_status ph_far_cross_check(int kernel, int d, int dtheta, int p_s, const int* degree, const double* s_lo,
                             const double* s_hi, const double* t_lo, const double* t_hi, const double* theta_lo,
                             const double* theta_hi, double eps, int cap, int* ranks, double* approx);

/* Fill *info with sizes and counts of a built handle. */
ph_status ph_get_info(const ph_handle* h, ph_info* info);

/* Serialise a handle (tree, block lists, all stored cores) to a file / rebuild a
 * handle from such a file on `device`.  ph_load reads and checks the whole file on the host
 * before it touches the device: every length against the bytes left in the file, and every
 * stored offset, index and size against the table or arena it points into; a file that
 * fails any check is refused with PH_ERR_IO (message in ph_last_error(NULL)), a missing
 * device gives PH_ERR_CUDA. */
ph_status ph_save(const ph_handle* h, const char* path);
ph_status ph_load(const char* path, int device, ph_handle** out);

/* Release every host and device resource of the handle; NULL is ignored. */
void ph_destroy(ph_handle* h);

/* Description of the last error on this handle (or of the last failed call
 * without a handle when h is NULL).  Never NULL; valid until the next call. */
const char* ph_last_error(const ph_handle* h);

/* Host-only planning (no GPU needed): builds the cluster tree (§3.2) and the
 * block cluster tree (§3.4) for the given points and reports their sizes.
 *   counts : host array of 8 longs receiving
 *            {nodes, leaves, near blocks, far blocks, far keys (dedup classes),
 *             sum of near n_s*n_t, max near blocks per leaf, depth}
 *   perm   : host array of n ints or NULL; receives, for each position of the
 *            cluster order, the original point index. */
ph_status ph_plan(const double* points, long n, int d, int l_max, double eta,
                  long* counts, int* perm);

/* The same for the adaptive cluster tree (§3.2 with a leaf-size stopping rule instead of a fixed
 * depth): a node is split while it holds more than leaf_size points and its level is below 20;
 * empty children are dropped.  The block tree then also has near blocks between a leaf and an
 * inner cluster (counted in counts[2] and counts[5]; counts[6] counts leaf x leaf blocks only) and
 * far blocks between clusters of different levels, whose translation classes are keyed by both
 * levels.  Planning only: ph_offline_build builds uniform trees. */
ph_status ph_plan_adaptive(const double* points, long n, int d, int leaf_size, double eta, long* counts, int* perm);

/* Every launch of the library also sits in an NVTX range named for its kind (and each
 * ph_instantiate / ph_matvec / ph_matvec_batched in one named for the call); without an
 * attached tool these are no-ops.
 * Per-kernel device time, measured with CUDA events recorded on the stream each
 * kernel is launched on (for roofline reports).  While enabled, every launch of
 * the library is bracketed by an event pair; ph_profile_read synchronises the
 * handle's streams and returns, for each of the PH_PROF_KINDS kernel kinds in
 * the order
 *   0 instantiate, 1 gather, 2 near, 3 upsweep_leaf, 4 transfer_up,
 *   5 coupling (the TT chain, or phase 1 of the explicit coupling), 6 transfer_down,
 *   7 far_h, 8 combine, 9 coupling phase 2 (explicit coupling),
 * the summed milliseconds and the number of launches since the last read (or
 * since enabling), then starts a new count.  ms and launches are host arrays of
 * PH_PROF_KINDS elements. */
#define PH_PROF_KINDS 10

/* ph_matvec runs its far-field chain on a second, high-priority stream concurrently with the
 * near field (enable = 1, the default).  enable = 0 runs every kernel in order on the caller's
 * stream, so that per-kernel times measured with ph_profile_read are those of each kernel on
 * its own (used for roofline reports; the result is the same). */
ph_status ph_set_overlap(ph_handle* h, int enable);

/* enable = 1: on FP32 handles, 8 < m <= 16 right-hand sides and p_s^d a multiple of 32, phase 1
 * of the explicit coupling runs on the tensor cores (tcgen05.mma kind::tf32 with 3xTF32 split
 * operands; every two 32-wide K chunks accumulate in tensor memory and are summed in FP32
 * registers); enable = 0 (the default) selects the CUDA-core kernel, which is faster at the
 * ranks of the 3-D Matern workloads (r' ~ 27..64: each 3xTF32 chunk takes 12 small MMAs whose
 * issue cost exceeds their arithmetic).  The tensor-core result differs from the CUDA-core one by FP32-level rounding (the
 * split drops the low x low product and the tensor cores accumulate in their own order).
 * Errors: PH_ERR_INVALID_ARG for a NULL handle.  Not in the paper: a kernel selection switch. */
ph_status ph_set_tensor_cores(ph_handle* h, int enable);
ph_status ph_profile_enable(ph_handle* h, int enable);
ph_status ph_profile_read(ph_handle* h, double* ms, long* launches);

/* Library version string. */
const char* ph_version(void);

/* Self-test of the device-side wait bound (the paper has no counterpart).  Runs one CTA on
 * `device` that waits on an mbarrier nothing arrives on, with the same bounded wait the
 * bulk-copy and tensor-core kernels use (about one second of the global timer).  The kernel
 * gives up, records it and returns, so the context stays usable.  Returns PH_ERR_TIMEOUT
 * (what a wait that ran out produces) and stores the seconds waited in *waited (may be
 * NULL); PH_ERR_INVALID_ARG for a device that does not exist; PH_ERR_CUDA if the launch or
 * copy failed (message in ph_last_error(NULL)).  Allocates and frees 16 bytes of device
 * memory; synchronous. */
ph_status ph_selftest_wait_bound(int device, double* waited);

#ifdef __cplusplus
}
#endif

#endif /* PH_H */
