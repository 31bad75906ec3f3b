/*
 * paradiag.h - C ABI of the GB300 (sm_103a) ParaDIAG step with the additive
 * element-wise Vanka multigrid of He & Liu, "A Vanka-type multigrid solver for
 * complex-shifted Laplacian systems from diagonalization-based parallel-in-time
 * algorithms" (arXiv 2203.11154).
 *
 * The problem (Sec. 1, eq. (1)): (B kron I_h + I_t kron A) u = f, with B = V D V^{-1}
 * and A the five-point Laplacian (1/h^2)[.,-1,.;-1,4,-1;.,-1,.] on the N x N interior
 * of the unit square, homogeneous Dirichlet values, h = 1/(N+1), N = 2^k - 1.
 * The step: g = (V^{-1} kron I_h) f, then the n independent shifted systems of eq. (2)
 * (A + lam_j I) z_j = g_j solved by multigrid (Sec. 3 components, smoother of
 * eq. (3)/(6)), then u = (V kron I_h) z.
 *
 * Conventions for every call:
 *   - Grid vectors are row-major [n][N][N] (shift or time index outermost), no
 *     padding, point (i,j) at i*N + j.  Complex values are interleaved (re, im)
 *     pairs of the context's working type: double for precision 0 (FP64), float for
 *     the FP32 multigrid of precision 1.  Real vectors of paradiag_solve are double.
 *   - Pointers named d_* are device pointers owned by the caller; h_* are host
 *     pointers owned by the caller.  The context owns all other device memory.
 *   - Calls are ordered on the context's CUDA stream.  Calls that return counts or
 *     residuals to the host synchronise that stream before returning.
 *   - Errors are returned as pd_status; nothing throws across the ABI.  After a
 *     PD_ERR_CUDA the context must be destroyed.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef PARADIAG_H
#define PARADIAG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pd_ctx pd_ctx;

typedef enum {
    PD_OK = 0,
    PD_ERR_ARG = 1,     /* invalid argument (sizes, NULL, unsupported option) */
    PD_ERR_CUDA = 2,    /* a CUDA runtime call failed or the extension is unusable */
    PD_ERR_NOMEM = 3,   /* device or pinned host allocation failed */
    PD_ERR_NOCONV = 4,  /* tolerance not reached within maxit / max_refine */
    PD_ERR_NAN = 5,     /* a residual norm became NaN or Inf */
    PD_ERR_SING = 6,    /* a coarsest-grid matrix is singular */
    PD_ERR_STATE = 7    /* call not valid for this context (e.g. no V given) */
} pd_status;

typedef struct {
    int cycle_gamma;   /* 1 = V-cycle, 2 = W-cycle (Sec. 3 uses W) */
    int nu1, nu2;      /* pre- and post-smoothing steps (Sec. 3 uses 1, 0) */
    int coarsest_n;    /* interior size of the coarsest grid, 1, 3, 7 or 15 (h0 = 1/(n+1)) */
    int maxit;         /* cycles per shifted solve */
    double tol;        /* precision 0: relative residual per shift;
                          precision 1: relative residual of eq. (1) */
    int omega_mode;    /* 0: 24/25 (Vanka) or 4/5 (Jacobi), Sec. 2.1 and Sec. 3;
                          1: LFA optimum of eq. (5) per shift and level;
                          2: the caller's table given to paradiag_setup */
    int precision;     /* 0: FP64 throughout; 1: FP32 cycles inside FP64 refinement */
    int smoother;      /* 0: additive element-wise Vanka (eq. (6)); 1: damped Jacobi */
    double inner_tol;  /* precision 1: relative residual of each inner FP32 solve */
    int max_refine;    /* precision 1: maximum refinement steps */
    int imag_check;    /* paradiag_solve: also form Im((V kron I) z) and report max |Im| */
    int inner_maxit;   /* precision 1: cycles per inner FP32 solve at most */
    double stall_ratio;/* precision 1: an inner solve also stops once a cycle reduces its
                          relative residual by less than this factor (FP32 rounding of z
                          bounds the attainable residual near cond(L) * 6e-8); 0 = off */
    int fused;         /* on the global-memory levels, fuse the last pre-smoothing step with
                          residual and restriction, and interpolation with the first
                          post-smoothing step (same arithmetic, fewer memory passes):
                          1 for the FP32 multigrid only (FP64 is bound by arithmetic, which
                          the recomputed halos increase), 2 always, 0 never */
    int tensor_transforms; /* precision 1, n <= 128, N >= 127: the time transforms as TF32x3
                          tensor-core GEMMs (tcgen05; for n > 64 the rows of the forward and
                          the K dimension of the inverse split over two CTAs, the inverse's
                          halves summed through distributed shared memory of a two-CTA
                          cluster); 0: FP32 CUDA-core products */
    int fused_variant; /* implementation of the fused kernels: 0 = warp-streaming strips
                          with the rows per segment chosen at set-up by timing them on the
                          context's own levels, 1 = TMA-staged shared-memory tiles, 2 = as 0
                          (warp streams: cp.async ring, shuffles) */
    double kappa;      /* diffusion coefficient scaling A in eq. (1): (B kron I + kappa I kron A);
                          the shifted systems become (kappa A + lam_j I) z = b (default 1) */
    int outer_maxit;   /* precision 0: FP64 correction steps on eq. (1) after the first solve,
                          u += P^{-1}(fhat - (B kron I + kappa I kron A) u), until the relative
                          residual of eq. (1) is <= tol (0 = the single solve).  When B is not
                          the matrix whose shifts and V were given (e.g. sequential backward
                          Euler with the alpha-circulant shifts), this is the ParaDIAG-II
                          outer iteration; the precision-1 refinement does the same. */
    int cuda_graphs;   /* 1: each multigrid cycle is captured once into a CUDA graph (per
                          kind of cycle and tolerance) and replayed, when the context's
                          stream is not the legacy default stream and profiling is off;
                          0: every kernel launched one by one (default 1) */
    int fx_residual;   /* precision 1 with a bidiagonal B: the refinement residual of eq. (1)
                          without FP64 instructions (stencil difference exact in fixed point,
                          three FP32 limbs, one scale per 16 x 128 tile and time step; the
                          other terms in float-float; more accurate than the FP64 formula);
                          likewise the residuals of the refined shifted solves (eq. (2), per
                          complex component); 0: FP64 (default 1) */
    int fft_transforms; /* 1: when V and V^{-1} given at set-up are those of the alpha-
                          circulant B (pd_alpha_circulant, to 1e-12) and n is a power of two
                          <= 128, the time transforms run as Gamma-weighted FFTs (both
                          precisions); 0: dense products (default 1) */
} pd_config;

/* Fills cfg with V(1,1), coarsest 3, maxit 100, tol 1e-10, omega_mode 1, FP64,
 * Vanka, inner_tol 1e-6, max_refine 12, imag_check 1, inner_maxit 2, stall_ratio 0.5,
 * fused 1, tensor_transforms 1, fused_variant 0, kappa 1, outer_maxit 0, cuda_graphs 1,
 * fx_residual 1, fft_transforms 1. */
void pd_config_default(pd_config *cfg);

/*
 * The alpha-circulant backward-Euler time matrix (a circulant-type B, Sec. 1):
 * B = (1/tau)(I - C_alpha), C_alpha the cyclic down-shift with alpha in the top-right
 * corner, and B = V D V^{-1} in closed form:
 *   lam_j = (1 - alpha^{1/n} e^{2 pi i (j-1)/n}) / tau,
 *   V = Gamma^{-1} Fbar, Fbar_{kj} = e^{-2 pi i (k-1)(j-1)/n}, V^{-1} = (1/n) F Gamma,
 *   Gamma = diag(alpha^{(k-1)/n}).
 * Outputs (host, caller-allocated, any may be NULL): h_B n*n real row-major,
 * h_shifts 2n doubles (re, im), h_V and h_Vinv 2*n*n doubles (row-major complex),
 * h_u0_coef n doubles (1/tau, 0, ..., 0: the initial value enters the first step).
 * Errors: PD_ERR_ARG for n < 1, tau <= 0 or alpha not in (0, 1].
 */
pd_status pd_alpha_circulant(int n, double tau, double alpha, double *h_B, double *h_shifts,
                             double *h_V, double *h_Vinv, double *h_u0_coef);

/*
 * The shifts and eigenvector matrices alone (the same closed form as pd_alpha_circulant):
 * h_shifts 2n doubles, h_V and h_Vinv 2*n*n doubles, complex interleaved (re, im), the
 * layout of a C99 double _Complex array; any may be NULL.  Errors as pd_alpha_circulant.
 */
pd_status pd_shifts_alpha_circulant(int n, double tau, double alpha, double *h_shifts, double *h_V,
                                    double *h_Vinv);

/*
 * The diagonalisation B = V D V^{-1} of a real time matrix (Sec. 1: it splits the
 * all-at-once system (1) into the shifted systems (2)), on the host: balancing by powers
 * of two, Householder reduction to Hessenberg form, complex Schur form by shifted QR
 * steps, eigenvectors by back substitution on the triangular factor, V^{-1} by
 * Gauss-Jordan elimination with partial pivoting.  For the boundary-value B of
 * Example 1 (eq. (9)), the quasi-BVM B of Example 2 (eq. (10)) or any diagonalisable B
 * with distinct eigenvalues.
 *   n        1 <= n <= 4096.   h_B  n*n doubles, row-major, real.
 *   h_shifts 2n doubles (re, im) of D, any order; h_V, h_Vinv 2*n*n doubles, complex
 *            row-major, the columns of V of unit 2-norm; any output may be NULL.
 * Host only (no GPU needed).  Errors: PD_ERR_ARG (n, NULL h_B), PD_ERR_SING (non-finite
 * B, no convergence of the QR steps, or V singular: B not diagonalisable in FP64),
 * PD_ERR_NOMEM.
 */
pd_status pd_diagonalize(int n, const double *h_B, double *h_shifts, double *h_V, double *h_Vinv);

/*
 * Creates a context for N x N grids and n shifts (Sec. 1, eq. (1)-(2)).
 *   N         interior points per side, 2^k - 1 with N >= cfg->coarsest_n.
 *   h         mesh step; must equal 1/(N+1) (the unit square).
 *   n         number of shifts / time steps, 1 <= n <= 128.
 *   h_shifts  2n doubles: lam_j (re, im); or NULL together with h_V and h_Vinv when
 *             h_B is given: the context then diagonalises B itself (pd_diagonalize).
 *   h_V, h_Vinv  2*n*n doubles each (complex row-major) or both NULL (then only the
 *             shifted-solve calls are valid, unless B alone is given).
 *   h_B       n*n real time matrix, row-major, or NULL.  Required by precision 1
 *             (the refinement residual uses B directly, never V).
 *   h_u0_coef n doubles or NULL (zeros): fhat_k = f_k + u0_coef[k] u0.
 *   h_omega   [n][levels] relaxation parameters for omega_mode 2, else NULL.
 *   cfg       options (NULL = pd_config_default).
 *   stream    the cudaStream_t every call of this context is ordered on (NULL = the
 *             legacy default stream).  The context never creates or destroys streams.
 * Setup runs on the host (shift tables, LFA, coarsest-grid inverses) and allocates
 * all device memory.  Errors: PD_ERR_ARG, PD_ERR_NOMEM, PD_ERR_CUDA, PD_ERR_SING (also:
 * B given alone could not be diagonalised).
 */
pd_status paradiag_setup(pd_ctx **ctx, int N, double h, int n, const double *h_shifts,
                         const double *h_V, const double *h_Vinv, const double *h_B,
                         const double *h_u0_coef, const double *h_omega,
                         const pd_config *cfg, void *stream);

/*
 * Context of the adjoint step (used to differentiate a solve): the transpose of eq. (1),
 * (B^T kron I_h + kappa I_t kron A) w = g, with B^T = V^{-H} conj(D) V^H, i.e. the shifted
 * systems (kappa A + conj(lam_j) I) of the same multigrid, transforms V^H and V^{-H}, B^T
 * for the refinement residual, no initial-value term, the forward context's options,
 * relaxation table and stream.  Errors: PD_ERR_STATE without V, as paradiag_setup.
 */
pd_status pd_adjoint_setup(const pd_ctx *ctx, pd_ctx **adj);

/* Number of grid levels (finest N down to the coarsest) and the relaxation
 * parameter table [n][levels] the context uses (host copy). */
int pd_num_levels(const pd_ctx *ctx);
pd_status pd_get_omega(const pd_ctx *ctx, double *h_omega);

/*
 * One multigrid cycle (Sec. 3: nu1 smoothing steps, full-weighting restriction of
 * the residual, gamma recursive cycles on the problem re-discretised at 2h with zero
 * initial guess, linear interpolation of the correction, nu2 smoothing steps) for all
 * n shifts at grid level `level` (0 = finest, N_l = (N_{l-1}-1)/2), in place:
 * d_z [n][N_l][N_l] holds the iterate on entry and on return; d_b the right-hand
 * side.  Working type per precision (see above).  Asynchronous.
 */
pd_status mg_vcycle(pd_ctx *ctx, int level, void *d_z, const void *d_b);

/*
 * Solves L_j z_j = b_j (eq. (2)) for all n shifts by cycles from z = 0 until
 * ||b_j - L_j z_j||_2 / ||b_j||_2 <= cfg.tol (checked before the first cycle and after
 * each one) or maxit cycles; converged shifts stop while others continue.
 * d_b, d_z: [n][N][N] complex of the working type.  h_iters, h_relres (n each, may be
 * NULL) receive cycles and final relative residual per shift.  Synchronises.
 * Returns PD_ERR_NOCONV if any shift missed the tolerance, PD_ERR_NAN on NaN/Inf.
 */
pd_status shifted_solve_batched(pd_ctx *ctx, void *d_z, const void *d_b, int *h_iters,
                                double *h_relres);

/*
 * The shifted systems of eq. (2), (kappa A + lam_j I) z_j = b_j, to the FP64 relative
 * residual cfg.tol per shift, with FP64 complex d_z, d_b [n][N][N] for either precision.
 * Precision 0: as shifted_solve_batched.  Precision 1: FP64 iterative refinement per shift
 * around the FP32 multigrid: r_j = b_j - L_j z_j in FP64, at most inner_maxit FP32 cycles
 * (stall_ratio as in paradiag_solve) for the correction, z_j += d_j in FP64; a shift stops
 * once its FP64 relative residual is <= tol, after max_refine corrections, or when a
 * correction reduces it by less than 10 %.  h_iters: FP32 cycles summed over corrections;
 * h_relres: the last FP64 relative residual.  Synchronises.  Errors: PD_ERR_NOCONV if a
 * shift missed tol, PD_ERR_NAN, PD_ERR_CUDA.
 */
pd_status shifted_solve_refined(pd_ctx *ctx, void *d_z, const void *d_b, int *h_iters,
                                double *h_relres);

/*
 * A batch of independent shifted-system problems of uneven sizes (several PDE instances,
 * each with its own grid N_i = 2^k - 1 and n_i shifts): one context per instance with the
 * common cfg (omega_mode 0 or 1; no V, B or tables).  pd_batch_solve advances all
 * instances together with the solve of shifted_solve_refined per instance.  With FP32
 * V(1,1) cycles (precision 1) every cycle of all instances runs as one launch per
 * multigrid level over all instances (see pd_batch_info), replayed as a CUDA graph when
 * cfg.cuda_graphs; otherwise each instance runs on a stream of its own that the batch
 * creates, one cycle of every unfinished instance per round, so that their kernels
 * overlap.  The solve is ordered after the work queued on `stream` before the call, and
 * work queued on `stream` after it waits for it.
 *   h_N, h_n: count sizes; h_shifts[i]: n_i complex shifts (host, copied).
 *   d_z[i], d_b[i]: FP64 complex [n_i][N_i][N_i] device arrays of instance i.
 *   h_iters, h_relres (may be NULL): sum n_i entries, instance by instance.
 * The paper has no multi-instance form: this batches the independent solves of eq. (2).
 * Errors: PD_ERR_ARG (count outside 1..64, a bad instance), the instance's setup or solve
 * error (the first in instance order; pd_batch_last_error gives its text).
 */
typedef struct pd_batch pd_batch;
pd_status pd_batch_setup(pd_batch **batch, int count, const int *h_N, const int *h_n,
                         const double *const *h_shifts, const pd_config *cfg, void *stream);
pd_status pd_batch_solve(pd_batch *batch, void *const *d_z, const void *const *d_b, int *h_iters,
                         double *h_relres);
pd_status pd_batch_destroy(pd_batch *batch);
const char *pd_batch_last_error(const pd_batch *batch);
/*
 * How a batch runs its cycles: *h_batched = 1 when every cycle of all instances is one
 * launch per multigrid level over all instances (FP32 V(1,1) cycles with the warp-stream
 * kernels, cfg.fused_variant 0 or 2: the instances share one stream, and a cycle is
 * 2 G + 2 launches, G the most global-memory levels of an instance, returned in
 * *h_launches_per_cycle), 0 when the instances run side by side on streams of their own
 * (-1 per cycle).  *h_launches: batched multigrid launches so far.  Any pointer may be NULL.
 */
pd_status pd_batch_info(const pd_batch *batch, int *h_batched, int *h_launches_per_cycle,
                        long long *h_launches);
/* Every kernel launch of the batch so far: the batched multigrid launches and those of the
 * instances' own evaluations (residuals, updates, norms); 0 for a NULL batch. */
long long pd_batch_launch_count(const pd_batch *batch);

/* Indices of the values paradiag_solve writes to h_stats (PD_STATS_LEN doubles). */
enum {
    PD_STAT_RELRES_ALLATONCE = 0, /* ||fhat - (B kron I + I kron A) u|| / ||fhat||, or -1 without B */
    PD_STAT_REFINE_STEPS = 1,     /* refinement steps (precision 1), 0 for FP64 */
    PD_STAT_IMAG_MAX = 2,         /* max |Im((V kron I) z)| of the last step (imag_check); -1
                                     where it is not formed (the tensor-core inverse, n > 64) */
    PD_STAT_CYCLES_TOTAL = 3,     /* multigrid cycles summed over shifts and steps */
    PD_STAT_CYCLES_MAX = 4,       /* max over shifts of cycles, summed over steps */
    PD_STAT_RELRES_SHIFT_MAX = 5, /* max over shifts of the last shifted relative residual */
    PD_STATS_LEN = 8
};

/*
 * One ParaDIAG solve of eq. (1) (device buffers):
 *   fhat_k = f_k + u0_coef[k] u0                      (right-hand side)
 *   g = (V^{-1} kron I_h) fhat                        (eq. (1))
 *   z_j = L_j^{-1} g_j by multigrid to cfg.tol        (eq. (2))
 *   u = Re (V kron I_h) z                             (eq. (1))
 * precision 1 wraps FP32 multigrid and compensated transforms in FP64 iterative
 * refinement on eq. (1) itself: r = fhat - (B kron I + I kron A) u in FP64, a step
 * above on r, u += d, until ||r|| / ||fhat|| <= cfg.tol.
 *   d_u   [n][N][N] double, output (precision 0 and 1).
 *   d_f   [n][N][N] double.   d_u0  [N][N] double (may be NULL: zero).
 *   h_iters/h_relres  per-shift cycles (summed over refinement steps) and last
 *                     relative residual, n each, may be NULL.
 *   h_stats           PD_STATS_LEN doubles, may be NULL.
 * Synchronises.  Errors: PD_ERR_STATE without V, PD_ERR_NOCONV, PD_ERR_NAN, CUDA.
 */
pd_status paradiag_solve(pd_ctx *ctx, double *d_u, const double *d_f, const double *d_u0,
                         int *h_iters, double *h_relres, double *h_stats);

/*
 * paradiag_solve on host buffers: copies h_f (and h_u0) to context-owned device
 * buffers with cudaMemcpyAsync on the context stream, solves, and copies u back to
 * h_u.  Pinned (page-locked) host memory gives full copy bandwidth; pageable memory
 * works but is slower.  Same outputs and errors as paradiag_solve.
 */
pd_status paradiag_solve_host(pd_ctx *ctx, double *h_u, const double *h_f, const double *h_u0,
                              int *h_iters, double *h_relres, double *h_stats);

/*
 * count independent steps of eq. (1) with host buffers, pipelined: the host-to-device copy
 * of step k+1's f and u0 and the device-to-host copy of step k-1's u run on two copy
 * streams (one per direction) that the context creates (once) while step k is solved on
 * the context's stream, through
 * two device staging sets (2 x (f, u, u0)).  Where h_u[k] is page-locked and 16-byte aligned
 * (and the array a multiple of 16 bytes), u goes out by a copy kernel of the library writing
 * the mapped host memory with streaming stores, which disturbs the concurrent solve less than
 * a copy-engine transfer; otherwise by the copy engine.  h_u[k], h_f[k]: [n][N][N] double host
 * arrays (pinned for full speed); h_u0 NULL or h_u0[k] NULL for no initial-value term.  h_iters,
 * h_relres: count x n entries; h_stats: count x PD_STATS_LEN (each may be NULL).
 * Synchronises.  Returns the first non-OK status of the steps (PD_ERR_CUDA at once).
 */
pd_status paradiag_solve_host_batch(pd_ctx *ctx, int count, double *const *h_u,
                                    const double *const *h_f, const double *const *h_u0,
                                    int *h_iters, double *h_relres, double *h_stats);

/*
 * Component entry points (one kernel each, all shifts of one level, asynchronous),
 * exposed so that each kernel can be checked against the oracle on its own.  Grid
 * arrays are [n][N_l][N_l] complex of the working type unless stated otherwise.
 *   pd_smooth             d_z_out = d_z_in + omega_{j,l} M_{e,j} (d_b - L_j d_z_in):
 *                         one step of S_j = I - omega M_{e,j} L_j (Sec. 2), stencil of
 *                         eq. (6); d_z_out must not alias d_z_in.
 *   pd_residual_restrict  d_bc [n][N_{l+1}]^2 = full weighting (Sec. 3) of
 *                         d_b - L_j d_z at grid level l.
 *   pd_prolong_add        d_z += linear interpolation (Sec. 3) of d_ec [n][N_{l+1}]^2.
 *   pd_coarse_solve       d_z = L_j^{-1} d_b on the coarsest level (inverse formed at
 *                         setup by Gauss-Jordan elimination with partial pivoting).
 *   pd_transform_forward  d_g = (V^{-1} kron I_h)(d_f + u0_coef kron d_u0), eq. (1):
 *                         d_f [n][N][N] double, d_u0 [N][N] double or NULL, d_g complex
 *                         of the working type.
 *   pd_transform_inverse  d_u = Re (V kron I_h) d_z (accumulate = 0) or
 *                         d_u += Re (V kron I_h) d_z (accumulate = 1), eq. (1): d_z
 *                         complex of the working type, d_u [n][N][N] double.
 *   pd_allatonce_residual d_r = fhat - (B kron I_h + I_t kron A) d_u, fhat as above,
 *                         in FP64 with the B given at setup; h_norms[0] = ||d_r||_2,
 *                         h_norms[1] = ||fhat||_2.  Synchronises.
 */
pd_status pd_smooth(pd_ctx *ctx, int level, void *d_z_out, const void *d_z_in, const void *d_b);
pd_status pd_residual_restrict(pd_ctx *ctx, int level, void *d_bc, const void *d_z,
                               const void *d_b);
pd_status pd_prolong_add(pd_ctx *ctx, int level, void *d_z, const void *d_ec);
pd_status pd_coarse_solve(pd_ctx *ctx, void *d_z, const void *d_b);
pd_status pd_transform_forward(pd_ctx *ctx, void *d_g, const double *d_f, const double *d_u0);
pd_status pd_transform_inverse(pd_ctx *ctx, double *d_u, const void *d_z, int accumulate);
pd_status pd_allatonce_residual(pd_ctx *ctx, double *d_r, const double *d_u, const double *d_f,
                                const double *d_u0, double *h_norms);

/*
 * The refinement's residual of eq. (1) as it is handed to the FP32 forward transform:
 * d_r32 [n][N][N] float = fhat - (B kron I_h + kappa I_t kron A) d_u rounded to FP32,
 * h_norms[0] = ||r||_2 (of the FP32 values), h_norms[1] = ||fhat||_2.  With a bidiagonal B
 * and cfg.fx_residual, computed without FP64 arithmetic (see fx_residual); else with the
 * FP64 formula.  Needs precision 1 and B (else PD_ERR_STATE).  Synchronises.
 */
pd_status pd_allatonce_residual32(pd_ctx *ctx, float *d_r32, const double *d_u, const double *d_f,
                                  const double *d_u0, double *h_norms);

/*
 * The residual of the shifted systems of eq. (2) as the refined shifted solves hand it to
 * the FP32 multigrid: d_r32 [n][N][N] complex float = b_j - (kappa A + lam_j I) z_j
 * rounded to FP32 (unscaled), h_norms[j] = ||r_j||_2 of the FP32 values (n doubles, may
 * be NULL).  d_z, d_b: [n][N][N] complex double, device.  With cfg.fx_residual the exact
 * stencil difference per complex component without FP64 arithmetic, else the FP64
 * formula.  Needs precision 1 (else PD_ERR_STATE).  Synchronises.
 */
pd_status pd_shifted_residual32(pd_ctx *ctx, float *d_r32, const void *d_z, const void *d_b,
                                double *h_norms);

/*
 * Gradient reduction of the adjoint (differentiation with respect to a coefficient
 * kappa scaling A in eq. (1)): *h_out = sum_k <d_w_k, A d_u_k>, A the five-point
 * operator of the context's grid (Sec. 1), in FP64 with a fixed summation order.
 * d_w, d_u: [n][N][N] double, device.  Synchronises.
 */
pd_status pd_laplacian_dot(pd_ctx *ctx, const double *d_w, const double *d_u, double *h_out);

/*
 * Gradient with respect to the initial value: fhat_k = f_k + u0_coef[k] u0, so
 * d_gu0 = sum_k u0_coef[k] d_w_k for the adjoint solution d_w (the forward context's
 * u0_coef).  d_w: [n][N][N] double, d_gu0: [N][N] double, device.  Asynchronous.
 */
pd_status pd_initial_value_gradient(pd_ctx *ctx, const double *d_w, double *d_gu0);

/*
 * Allocation-free residual check for the alpha-circulant backward-Euler system (the
 * paper has no counterpart; it is a service for callers of this library).
 *
 * For callers that cannot call cudaMalloc where they need this check - a framework that
 * owns all device memory through its own pool or arena and forbids other allocations,
 * or a time-critical loop that cannot afford cudaMalloc's device-wide synchronisation.
 * It needs no context and allocates nothing: the caller passes every input and output,
 * and the only scratch (per-CTA partial sums) lives in a fixed 128 KiB array in device
 * memory inside the library, which every GPU that loads the library keeps until exit.
 *
 * Computes, for B = (1/tau)(I - C_alpha) and fhat_1 = f_1 + u0 / tau, fhat_k = f_k else:
 *   d_r = fhat - (B kron I_h + I_t kron A) d_u      (d_r may be NULL: norms only)
 *   d_norms[0] = ||d_r||_2,  d_norms[1] = ||fhat||_2   (two doubles, device memory)
 * d_u, d_f, d_r: [n][N][N] double, device; d_u0: [N][N] double or NULL; stream: the
 * cudaStream_t the two kernels run on (NULL = legacy default stream).  Asynchronous.
 * Limits: n <= 128 (the size of the scratch array); larger n returns PD_ERR_ARG, as do
 * N < 1, tau <= 0, alpha outside (0, 1] and NULL d_u, d_f or d_norms.
 * The first call on a device looks up the scratch array's device address (with that
 * device current) and caches it; make that first call before any stream capture.
 * All calls share the scratch array: calls whose kernels may overlap on the GPU (on
 * different streams without ordering between them) race and must not be issued.
 */
pd_status pd_allatonce_residual_static(int N, int n, double tau, double alpha, const double *d_u,
                                       const double *d_f, const double *d_u0, double *d_r,
                                       double *d_norms, void *stream);

/*
 * Instrumentation (no counterpart in the paper).  While enabled, the context records a
 * CUDA event pair on its stream around every kernel launch and attributes it to one of
 * the classes below, together with the algorithmic bytes of the launch (each array
 * element read or written once, counting only shifts that are still iterating).
 * pd_profile_enable(ctx, 1) clears the totals; pd_profile_read synchronises and
 * returns the totals of one class (any output pointer may be NULL).
 */
enum {
    PD_KC_SMOOTH0 = 0,   /* smoothing steps on the finest grid */
    PD_KC_RESTRICT0 = 1, /* residual + full weighting from the finest grid */
    PD_KC_PROLONG0 = 2,  /* interpolation + correction on the finest grid */
    PD_KC_SMOOTH_C = 3,  /* the same three on the other global-memory levels */
    PD_KC_RESTRICT_C = 4,
    PD_KC_PROLONG_C = 5,
    PD_KC_COARSE = 6,    /* coarse levels and coarsest solve, one CTA per shift */
    PD_KC_CONVERGE = 7,  /* per-shift convergence test */
    PD_KC_FORWARD = 8,   /* (V^{-1} kron I_h) */
    PD_KC_INVERSE = 9,   /* (V kron I_h) */
    PD_KC_RESIDUAL = 10, /* FP64 residual of eq. (1) */
    PD_KC_OTHER = 11,    /* copies, state reset */
    PD_KC_SR0 = 12,      /* fused smoothing + residual + restriction, finest grid */
    PD_KC_PS0 = 13,      /* fused interpolation + smoothing, finest grid */
    PD_KC_SR_C = 14,     /* the same two on the other global-memory levels */
    PD_KC_PS_C = 15,
    PD_KC_COUNT = 16
};
pd_status pd_profile_enable(pd_ctx *ctx, int on);
pd_status pd_profile_read(pd_ctx *ctx, int kclass, double *total_ms, long long *launches,
                          double *alg_bytes);

/*
 * Convergence history of the last solve (the paper reports reductions of the relative
 * residual, Sec. 3; no call of its own).  Synchronises.
 *   h_cycle_len [n], h_cycle_hist [n][cap]: per shift, the relative residual of eq. (2)
 *     before the first cycle and after each cycle of the last multigrid solve (for the
 *     precision form: its last inner FP32 solve; for shifted_solve_refined: the last
 *     correction's inner solve); entries beyond h_cycle_len[j] are 0, and -1 marks an
 *     iterate whose residual was not formed (an inner solve's last cycle: the refinement
 *     evaluates the residual of eq. (1) instead).
 *   h_outer_len, h_outer [cap_outer]: the relative residual of eq. (1) after each
 *     refinement (precision 1) or correction (outer_maxit) step of the last paradiag_solve.
 * Any output pointer may be NULL.  Errors: PD_ERR_ARG (cap < 0), PD_ERR_CUDA.
 */
pd_status pd_get_history(pd_ctx *ctx, int cap, int *h_cycle_len, double *h_cycle_hist,
                         int cap_outer, int *h_outer_len, double *h_outer);

/* Waits for the context stream. */
pd_status pd_synchronize(pd_ctx *ctx);

/* Kernel launches issued by this context since creation (for launch accounting). */
long long pd_launch_count(const pd_ctx *ctx);

/*
 * The fused smoothing kernels the set-up autotuner chose for multigrid level `level` (0 =
 * finest) of the working precision: *h_variant = 1 (TMA tiles), 2 (warp streams, *h_seg
 * rows per segment) or 0 where the level has no fused kernels (levels held in one CTA per
 * shift, the last level, cfg.fused = 0, the FP64 form with cfg.fused = 1).  Errors: PD_ERR_ARG (NULL ctx, level outside
 * 0..levels-1).  Instrumentation; the paper has no counterpart.
 */
pd_status pd_fused_choice(const pd_ctx *ctx, int level, int *h_variant, int *h_seg);

/* Waits for the context stream, then frees all device and pinned host memory of the
 * context. */
pd_status paradiag_destroy(pd_ctx *ctx);

/* Static description of a status code. */
const char *pd_status_str(pd_status s);

/* Text of the last error recorded in the context (CUDA error string or argument). */
const char *pd_last_error(const pd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PARADIAG_H */
