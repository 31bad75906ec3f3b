/*
 * FP64 complex CPU oracle for the ParaDIAG step with the additive element-wise
 * Vanka multigrid of He & Liu, "A Vanka-type multigrid solver for complex-shifted
 * Laplacian systems from diagonalization-based parallel-in-time algorithms".
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It is plain, slow, obviously
 * correct C: every grid operation is a loop over points with explicit zero
 * Dirichlet values outside the interior, every step follows the paper's order, and
 * nothing is blocked, fused or reordered.  It shares no code, header or table with
 * the CUDA path.
 *
 * Conventions:
 *   - A level has N x N interior points, N = 2^k - 1, mesh step h = 1/(N+1);
 *     arrays are row-major [N][N], point (i,j) at i*N + j.
 *   - Coarse point (ci,cj) of the next level sits on fine point (2ci+1, 2cj+1).
 *   - The only parallelism is OpenMP over independent shifts / time rows; each
 *     loop body is the plain definition.
 *
 * Parity status: every function below is pinned by a CPU test (closed forms,
 * dense solves, brute-force patch sums, Table 1, manufactured solutions, the
 * all-at-once residual of eq. (1)), except the iteration counts per shift, whose
 * published values (Figures 1-3) are not available: those are "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_PI 3.14159265358979323846

/* value of a level array with the zero Dirichlet extension outside the interior */
static cplx at(const cplx *v, int N, int i, int j)
{
    if (i < 0 || i >= N || j < 0 || j >= N)
        return 0.0;
    return v[(size_t)i * N + j];
}

/* out = (A + lam I) z, A the five-point Laplacian (1/h^2)[.,-1,.;-1,4,-1;.,-1,.]
 * with homogeneous Dirichlet values (Sec. 1, eq. (2) and the stencil after it). */
void or_apply_shifted_laplacian(int N, double h, cplx lam, const cplx *z, cplx *out)
{
    double ih2 = 1.0 / (h * h);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            cplx lap = 4.0 * at(z, N, i, j) - at(z, N, i - 1, j) - at(z, N, i + 1, j)
                       - at(z, N, i, j - 1) - at(z, N, i, j + 1);
            out[(size_t)i * N + j] = ih2 * lap + lam * at(z, N, i, j);
        }
}

/* r = b - L_j z  (eq. (2)) */
void or_residual(int N, double h, cplx lam, const cplx *b, const cplx *z, cplx *r)
{
    size_t m = (size_t)N * N;
    or_apply_shifted_laplacian(N, h, lam, z, r);
    for (size_t p = 0; p < m; p++)
        r[p] = b[p] - r[p];
}

/* a, b, c of the explicit element-wise Vanka stencil, eq. (6), eta = lam h^2 */
void or_vanka_abc(cplx eta, cplx *a, cplx *b, cplx *c)
{
    cplx p = 1.0 / (2.0 + eta);
    cplx q = 1.0 / (4.0 + eta);
    cplx s = 1.0 / (6.0 + eta);
    *a = 0.25 * (p + 2.0 * q + s);
    *b = 0.25 * (p - s);
    *c = 0.25 * (p - 2.0 * q + s);
}

/* One relaxation step S_j = I - omega M_{e,j} L_j (Sec. 2): z <- z + omega M r with
 * r = b - L_j z computed in full first (additive smoother: every update uses the
 * old z).  M is the stencil (h^2/4)[c,2b,c; 2b,4a,2b; c,2b,c] of eq. (6) applied at
 * every interior point, residual values outside the interior taken as zero. */
void or_vanka_smooth(int N, double h, cplx lam, double omega, const cplx *b, cplx *z)
{
    size_t m = (size_t)N * N;
    cplx *r = malloc(m * sizeof(cplx));
    or_residual(N, h, lam, b, z, r);
    cplx a, bb, c;
    or_vanka_abc(lam * h * h, &a, &bb, &c);
    double s4 = h * h / 4.0;
    cplx w[3][3] = {{s4 * c, s4 * 2.0 * bb, s4 * c},
                    {s4 * 2.0 * bb, s4 * 4.0 * a, s4 * 2.0 * bb},
                    {s4 * c, s4 * 2.0 * bb, s4 * c}};
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            cplx s = 0.0;
            for (int di = -1; di <= 1; di++)
                for (int dj = -1; dj <= 1; dj++)
                    s += w[di + 1][dj + 1] * at(r, N, i + di, j + dj);
            z[(size_t)i * N + j] += omega * s;
        }
    free(r);
}

/* Damped point Jacobi, M = D^{-1} = h^2/(4+eta) I, the comparison smoother of
 * Sec. 3 (omega = 4/5 there). */
void or_jacobi_smooth(int N, double h, cplx lam, double omega, const cplx *b, cplx *z)
{
    size_t m = (size_t)N * N;
    cplx *r = malloc(m * sizeof(cplx));
    or_residual(N, h, lam, b, z, r);
    cplx dinv = h * h / (4.0 + lam * h * h);
    for (size_t p = 0; p < m; p++)
        z[p] += omega * dinv * r[p];
    free(r);
}

/* Full-weighting restriction (Sec. 3): rc(ci,cj) = (1/16) sum w r(2ci+1+di, 2cj+1+dj),
 * w = [1 2 1; 2 4 2; 1 2 1]. */
static const double FW[3][3] = {{1, 2, 1}, {2, 4, 2}, {1, 2, 1}};

void or_restrict_fw(int Nf, const cplx *rf, cplx *rc)
{
    int Nc = (Nf - 1) / 2;
    for (int ci = 0; ci < Nc; ci++)
        for (int cj = 0; cj < Nc; cj++) {
            cplx s = 0.0;
            for (int di = -1; di <= 1; di++)
                for (int dj = -1; dj <= 1; dj++)
                    s += FW[di + 1][dj + 1] * at(rf, Nf, 2 * ci + 1 + di, 2 * cj + 1 + dj);
            rc[(size_t)ci * Nc + cj] = s / 16.0;
        }
}

/* Linear (bilinear) interpolation and correction (Sec. 3): zf += P ec with
 * P = 4 R^T, written as the scatter of each coarse value to its 3x3 fine
 * neighbourhood with weights w/4. */
void or_prolong_add(int Nf, const cplx *ec, cplx *zf)
{
    int Nc = (Nf - 1) / 2;
    for (int ci = 0; ci < Nc; ci++)
        for (int cj = 0; cj < Nc; cj++)
            for (int di = -1; di <= 1; di++)
                for (int dj = -1; dj <= 1; dj++)
                    zf[(size_t)(2 * ci + 1 + di) * Nf + (2 * cj + 1 + dj)] +=
                        FW[di + 1][dj + 1] / 4.0 * ec[(size_t)ci * Nc + cj];
}

/* Dense LU with partial pivoting, then forward and back substitution: solves
 * A x = rhs in place (A is m x m row-major and is overwritten).  Returns 0, or -1
 * for an exactly singular pivot. */
int or_dense_solve(int m, cplx *A, cplx *x)
{
    for (int k = 0; k < m; k++) {
        int p = k;
        for (int i = k + 1; i < m; i++)
            if (cabs(A[(size_t)i * m + k]) > cabs(A[(size_t)p * m + k]))
                p = i;
        if (A[(size_t)p * m + k] == 0.0)
            return -1;
        if (p != k) {
            for (int j = 0; j < m; j++) {
                cplx t = A[(size_t)k * m + j];
                A[(size_t)k * m + j] = A[(size_t)p * m + j];
                A[(size_t)p * m + j] = t;
            }
            cplx t = x[k];
            x[k] = x[p];
            x[p] = t;
        }
        for (int i = k + 1; i < m; i++) {
            cplx l = A[(size_t)i * m + k] / A[(size_t)k * m + k];
            A[(size_t)i * m + k] = l;
            for (int j = k + 1; j < m; j++)
                A[(size_t)i * m + j] -= l * A[(size_t)k * m + j];
            x[i] -= l * x[k];
        }
    }
    for (int k = m - 1; k >= 0; k--) {
        cplx s = x[k];
        for (int j = k + 1; j < m; j++)
            s -= A[(size_t)k * m + j] * x[j];
        x[k] = s / A[(size_t)k * m + k];
    }
    return 0;
}

/* Coarsest-grid direct solve: z = L_j^{-1} b by dense LU of the assembled matrix
 * (the coarsest grid of Sec. 3).  Column q of the matrix is L_j applied to e_q. */
int or_coarse_solve(int N, double h, cplx lam, const cplx *b, cplx *z)
{
    int m = N * N;
    cplx *Amat = malloc((size_t)m * m * sizeof(cplx));
    cplx *e = calloc((size_t)m, sizeof(cplx));
    cplx *col = malloc((size_t)m * sizeof(cplx));
    for (int q = 0; q < m; q++) {
        e[q] = 1.0;
        or_apply_shifted_laplacian(N, h, lam, e, col);
        e[q] = 0.0;
        for (int p = 0; p < m; p++)
            Amat[(size_t)p * m + q] = col[p];
    }
    memcpy(z, b, (size_t)m * sizeof(cplx));
    int rc = or_dense_solve(m, Amat, z);
    free(Amat);
    free(e);
    free(col);
    return rc;
}

/* Multigrid parameters: cycle index gamma (1 = V, 2 = W), nu1 pre- and nu2
 * post-smoothing steps, the interior size of the coarsest grid, and the smoother
 * (0 = additive Vanka of eq. (6), 1 = damped Jacobi). */
typedef struct {
    int gamma, nu1, nu2, coarsest_n, smoother;
} or_mg_params;

static void smooth(const or_mg_params *prm, int N, double h, cplx lam, double omega,
                   const cplx *b, cplx *z)
{
    if (prm->smoother == 1)
        or_jacobi_smooth(N, h, lam, omega, b, z);
    else
        or_vanka_smooth(N, h, lam, omega, b, z);
}

/* One multigrid cycle on the level with N interior points (Sec. 3: coarse
 * operators re-discretised at 2h, full weighting, linear interpolation, gamma
 * recursive calls).  omega[l] is the relaxation parameter of level l, counted from
 * this level. */
int or_mg_cycle(const or_mg_params *prm, int N, cplx lam, const double *omega,
                const cplx *b, cplx *z)
{
    double h = 1.0 / (N + 1);
    if (N <= prm->coarsest_n)
        return or_coarse_solve(N, h, lam, b, z);
    for (int s = 0; s < prm->nu1; s++)
        smooth(prm, N, h, lam, omega[0], b, z);
    int Nc = (N - 1) / 2;
    size_t m = (size_t)N * N, mc = (size_t)Nc * Nc;
    cplx *r = malloc(m * sizeof(cplx));
    cplx *bc = malloc(mc * sizeof(cplx));
    cplx *ec = calloc(mc, sizeof(cplx));
    or_residual(N, h, lam, b, z, r);
    or_restrict_fw(N, r, bc);
    int rc = 0;
    for (int g = 0; g < prm->gamma && rc == 0; g++)
        rc = or_mg_cycle(prm, Nc, lam, omega + 1, bc, ec);
    or_prolong_add(N, ec, z);
    for (int s = 0; s < prm->nu2; s++)
        smooth(prm, N, h, lam, omega[0], b, z);
    free(r);
    free(bc);
    free(ec);
    return rc;
}

static double norm2(size_t m, const cplx *v)
{
    double s = 0.0;
    for (size_t p = 0; p < m; p++)
        s += creal(v[p]) * creal(v[p]) + cimag(v[p]) * cimag(v[p]);
    return sqrt(s);
}

/* Solve L_j z = b_j (eq. (2)) by cycles from z = 0 until the relative residual
 * ||b - L_j z||_2 / ||b||_2 is at most tol, checked before the first and after each
 * cycle, or maxit cycles are done.  Returns the cycles done in *iters and the last
 * relative residual in *relres; hist (may be NULL) receives relres after 0..iters
 * cycles.  b = 0 gives z = 0, iters = 0, relres = 0. */
int or_shifted_solve(const or_mg_params *prm, int N, cplx lam, const double *omega,
                     int maxit, double tol, const cplx *b, cplx *z, int *iters,
                     double *relres, double *hist)
{
    size_t m = (size_t)N * N;
    double h = 1.0 / (N + 1);
    memset(z, 0, m * sizeof(cplx));
    double bn = norm2(m, b);
    *iters = 0;
    *relres = 0.0;
    if (bn == 0.0) {
        if (hist)
            hist[0] = 0.0;
        return 0;
    }
    cplx *r = malloc(m * sizeof(cplx));
    int k = 0, rc = 0;
    for (;;) {
        or_residual(N, h, lam, b, z, r);
        double rr = norm2(m, r) / bn;
        if (hist)
            hist[k] = rr;
        *relres = rr;
        if (rr <= tol || k >= maxit || rc != 0)
            break;
        rc = or_mg_cycle(prm, N, lam, omega, b, z);
        k++;
    }
    *iters = k;
    free(r);
    return rc;
}

/* The n shifted solves of eq. (2), independent, one OpenMP task per shift.
 * b, z: [n][N][N]; omega: [n][levels]; iters, relres: [n]. */
int or_shifted_solve_batch(const or_mg_params *prm, int N, int n, const cplx *lam,
                           const double *omega, int levels, int maxit, double tol,
                           const cplx *b, cplx *z, int *iters, double *relres)
{
    size_t m = (size_t)N * N;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int j = 0; j < n; j++)
        bad |= (or_shifted_solve(prm, N, lam[j], omega + (size_t)j * levels, maxit, tol,
                                 b + j * m, z + j * m, &iters[j], &relres[j], NULL) != 0);
    return bad ? -1 : 0;
}

/* alpha-circulant backward-Euler time matrix B = (1/tau)(I - C_alpha), C_alpha the
 * cyclic down-shift with alpha in the top-right corner (a circulant-type B, Sec. 1),
 * and its diagonalisation B = V D V^{-1}:
 *   lam_j = (1 - alpha^{1/n} e^{2 pi i (j-1)/n}) / tau,
 *   V = Gamma^{-1} Fbar,  Fbar_{kj} = e^{-2 pi i (k-1)(j-1)/n},
 *   V^{-1} = (1/n) F Gamma,  Gamma = diag(alpha^{(k-1)/n}).
 * Zero-based indices below; V and Vinv are n x n row-major. */
void or_alpha_circulant(int n, double tau, double alpha, cplx *lam, cplx *V, cplx *Vinv)
{
    double an = pow(alpha, 1.0 / n);
    for (int j = 0; j < n; j++)
        lam[j] = (1.0 - an * cexp(2.0 * OR_PI * I * j / n)) / tau;
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++) {
            V[(size_t)k * n + j] = pow(alpha, -(double)k / n) * cexp(-2.0 * OR_PI * I * k * j / n);
            Vinv[(size_t)k * n + j] = cexp(2.0 * OR_PI * I * k * j / n) * pow(alpha, (double)j / n) / n;
        }
}

/* Right-hand side of eq. (1) for backward Euler with initial value u0:
 * fhat_k = f_k, plus u0 / tau in the first time step. */
void or_assemble_rhs(int N, int n, double tau, const double *f, const double *u0, double *fhat)
{
    size_t m = (size_t)N * N;
    memcpy(fhat, f, (size_t)n * m * sizeof(double));
    for (size_t p = 0; p < m; p++)
        fhat[p] += u0[p] / tau;
}

/* y[j] = sum_k W[j][k] x[k] for every grid point: the (W kron I_h) product of
 * eq. (1) with W = V^{-1} or V; x, y are [n][m] complex. */
void or_time_transform(int n, size_t m, const cplx *W, const cplx *x, cplx *y)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; j++) {
        cplx *yj = y + (size_t)j * m;
        for (size_t p = 0; p < m; p++)
            yj[p] = 0.0;
        for (int k = 0; k < n; k++) {
            cplx w = W[(size_t)j * n + k];
            const cplx *xk = x + (size_t)k * m;
            for (size_t p = 0; p < m; p++)
                yj[p] += w * xk[p];
        }
    }
}

/* One ParaDIAG step for eq. (1): g = (V^{-1} kron I_h) fhat, z_j = L_j^{-1} g_j by
 * multigrid (eq. (2)), u = (V kron I_h) z.  fhat: [n][N][N] real; u: [n][N][N]
 * real part of the result; *imag_max receives max |Im|; iters/relres per shift. */
int or_paradiag_solve(const or_mg_params *prm, int N, int n, const cplx *lam, const cplx *V,
                      const cplx *Vinv, const double *omega, int levels, int maxit, double tol,
                      const double *fhat, double *u, double *imag_max, int *iters,
                      double *relres)
{
    size_t m = (size_t)N * N, nm = (size_t)n * m;
    cplx *x = malloc(nm * sizeof(cplx));
    cplx *g = malloc(nm * sizeof(cplx));
    cplx *z = malloc(nm * sizeof(cplx));
    for (size_t p = 0; p < nm; p++)
        x[p] = fhat[p];
    or_time_transform(n, m, Vinv, x, g);
    int rc = or_shifted_solve_batch(prm, N, n, lam, omega, levels, maxit, tol, g, z, iters,
                                    relres);
    or_time_transform(n, m, V, z, x);
    double im = 0.0;
    for (size_t p = 0; p < nm; p++) {
        u[p] = creal(x[p]);
        if (fabs(cimag(x[p])) > im)
            im = fabs(cimag(x[p]));
    }
    *imag_max = im;
    free(x);
    free(g);
    free(z);
    return rc;
}

/* Residual of the all-at-once system (1) for the alpha-circulant B, computed from
 * the sparse B directly (never through V):
 *   r_k = fhat_k - (u_k - u_{k-1}) / tau - A u_k,  with u_0 := alpha u_n.
 * Writes r (may be NULL) and returns ||r||_2; *fnorm receives ||fhat||_2. */
double or_allatonce_residual(int N, int n, double tau, double alpha, const double *u,
                             const double *fhat, double *r, double *fnorm)
{
    size_t m = (size_t)N * N;
    double h = 1.0 / (N + 1), ih2 = 1.0 / (h * h);
    double rs = 0.0, fs = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rs, fs)
    for (int k = 0; k < n; k++) {
        const double *uk = u + (size_t)k * m;
        const double *up = (k == 0) ? u + (size_t)(n - 1) * m : u + (size_t)(k - 1) * m;
        double cprev = (k == 0) ? alpha : 1.0;
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                size_t p = (size_t)i * N + j;
                double c = uk[p];
                double nb = (i > 0 ? uk[p - N] : 0.0) + (i < N - 1 ? uk[p + N] : 0.0)
                            + (j > 0 ? uk[p - 1] : 0.0) + (j < N - 1 ? uk[p + 1] : 0.0);
                double Au = ih2 * (4.0 * c - nb);
                double Bu = (c - cprev * up[p]) / tau;
                double rv = fhat[(size_t)k * m + p] - Bu - Au;
                if (r)
                    r[(size_t)k * m + p] = rv;
                rs += rv * rv;
                fs += fhat[(size_t)k * m + p] * fhat[(size_t)k * m + p];
            }
    }
    *fnorm = sqrt(fs);
    return sqrt(rs);
}

/* The same residual of eq. (1) (alpha-circulant backward Euler, unscaled A) evaluated in
 * long double (64-bit significand on x86-64, 113-bit on AArch64 Linux), each term formed
 * separately: a reference for residual kernels whose error lies below the FP64 rounding
 * of the formula.  r (may be NULL) receives the residual rounded to double. */
double or_allatonce_residual_ld(int N, int n, double tau, double alpha, const double *u,
                                const double *fhat, double *r)
{
    size_t m = (size_t)N * N;
    long double h = 1.0L / (N + 1), ih2 = 1.0L / (h * h);
    double rs = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rs)
    for (int k = 0; k < n; k++) {
        const double *uk = u + (size_t)k * m;
        const double *up = (k == 0) ? u + (size_t)(n - 1) * m : u + (size_t)(k - 1) * m;
        long double cprev = (k == 0) ? (long double)alpha : 1.0L;
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                size_t p = (size_t)i * N + j;
                long double c = uk[p];
                long double nb = (long double)(i > 0 ? uk[p - N] : 0.0) + (long double)(i < N - 1 ? uk[p + N] : 0.0)
                                 + (long double)(j > 0 ? uk[p - 1] : 0.0) + (long double)(j < N - 1 ? uk[p + 1] : 0.0);
                long double Au = ih2 * (4.0L * c - nb);
                long double Bu = (c - cprev * (long double)up[p]) / (long double)tau;
                long double rv = (long double)fhat[(size_t)k * m + p] - Bu - Au;
                if (r)
                    r[(size_t)k * m + p] = (double)rv;
                rs += (double)(rv * rv);
            }
    }
    return sqrt(rs);
}

/* r = b - (A + lam I) z of one shifted system (eq. (2)) evaluated in long double, each
 * component and term separately (a reference for residual kernels whose error lies below
 * the FP64 rounding of the formula); r receives the residual rounded to double, the
 * return value is ||r||_2 of the rounded values.  b, z, r: N x N complex. */
double or_residual_ld(int N, double h, cplx lam, const cplx *b, const cplx *z, cplx *r)
{
    long double ih2 = 1.0L / ((long double)h * (long double)h);
    long double lr = creal(lam), li = cimag(lam);
    double rs = 0.0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            size_t p = (size_t)i * N + j;
            long double cr = creal(z[p]), ci = cimag(z[p]);
            long double nr = (long double)creal(at(z, N, i - 1, j)) + (long double)creal(at(z, N, i + 1, j))
                             + (long double)creal(at(z, N, i, j - 1)) + (long double)creal(at(z, N, i, j + 1));
            long double ni = (long double)cimag(at(z, N, i - 1, j)) + (long double)cimag(at(z, N, i + 1, j))
                             + (long double)cimag(at(z, N, i, j - 1)) + (long double)cimag(at(z, N, i, j + 1));
            long double rr = (long double)creal(b[p]) - (lr * cr - li * ci) - ih2 * (4.0L * cr - nr);
            long double ri = (long double)cimag(b[p]) - (lr * ci + li * cr) - ih2 * (4.0L * ci - ni);
            r[p] = (double)rr + I * (double)ri;
            rs += (double)rr * (double)rr + (double)ri * (double)ri;
        }
    return sqrt(rs);
}

/* OpenMP thread count used by the batched routines (reported with CPU timings). */
void or_set_threads(int k)
{
    omp_set_num_threads(k);
}

int or_max_threads(void)
{
    return omp_get_max_threads();
}
