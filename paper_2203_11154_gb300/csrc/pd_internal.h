// Internal declarations shared by the translation units of libparadiag.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/paradiag.h"

namespace pd {

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarseDepth = 7;  // levels below the first one of the coarse CTA kernel
constexpr int kMaxShifts = 128;

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

// A strided grid array: element (shift j, row i, col c) at p[j*plane + i*pitch + c].
struct View {
  void *p;
  long long pitch;
  long long plane;
};

// Smoother coefficients of one (level, shift) in the h^2-scaled form used by every
// kernel: with rt = h^2 (b - L z) = h^2 b - d z + (sum of the 4 neighbours of z),
//   Vanka (eq. (6)):  z += ca rt + cb (sum of 4 edge neighbours of rt)
//                             + cc (sum of 4 corner neighbours of rt),
//   with d = 4 + eta, ca = omega a, cb = omega b / 2, cc = omega c / 4;
//   Jacobi: ca = omega / (4 + eta), cb = cc = 0.
template <typename T> struct Coef {
  typename Cx<T>::type d, ca, cb, cc;
};

// Per-shift state of a batched solve, device resident.
struct SolveState {
  int *active;        // [n] 1 while the shift still iterates
  int *iters;         // [n] cycles done
  int *final_buf;     // [n] ping-pong index holding the answer of level 0
  int *nactive;       // [1] number of active shifts
  int *flags;         // [1] bit 0: NaN/Inf seen
  double *bn2;        // [n] ||b_j||^2 (scaled)
  double *relres;     // [n] last relative residual
  double *partials;   // [n][max_tiles] per-CTA squared residual sums
  int max_tiles;
  double *hist;       // [n][hist_stride] relative residual before the first cycle and
  int hist_stride;    // after each one (entry k = after k cycles), or NULL
};

// ---- multigrid kernels (mg_kernels.cu), T = double or float ----
template <typename T>
void launch_smooth(cudaStream_t s, int N, int n, View zin, View zout, View b, T bscale,
                   const Coef<T> *coef, const int *active, bool z_zero, bool jacobi,
                   double *partials, int part_stride);
template <typename T>
void launch_resnorm(cudaStream_t s, int N, int n, View z, View b, T bscale, const Coef<T> *coef,
                    const int *active, bool z_zero, double *partials, int part_stride);
int smooth_tiles(int N);
void launch_reset_state(cudaStream_t s, int n, SolveState st);
void launch_finalize(cudaStream_t s, int n, SolveState st, int cur_buf);
void launch_converge(cudaStream_t s, int n, int ntiles, SolveState st, double tol, int maxit,
                     double stall, int cur_buf);
template <typename T>
void launch_residual_restrict(cudaStream_t s, int Nf, int n, View z, View b, T bscale, View bc,
                              T oscale, const Coef<T> *coef, const int *active, bool z_zero);
template <typename T>
void launch_prolong_add(cudaStream_t s, int Nf, int n, View z, View ec, const int *active);

// ---- time transforms by FFT for the alpha-circulant B (fft_transforms.cu) ----
bool fft_transforms_supported(int n);
template <typename T> cudaError_t prepare_fft_transforms();
template <typename T>
void launch_fft_forward(cudaStream_t s, int num_sms, int N, int n, View g, const void *f, bool f32,
                        const double *u0, const double *u0coef, const T *wk,
                        const typename Cx<T>::type *tw);
template <typename T>
void launch_fft_inverse(cudaStream_t s, int num_sms, int N, int n, double *u, View z0, View z1,
                        const int *final_buf, const T *wk, const typename Cx<T>::type *tw,
                        T dscale, bool accumulate, bool imag_check, unsigned long long *imag_bits);

// ---- residual of eq. (1) without FP64 arithmetic (residual_ws.cu) ----
// CTAs of one residual: the interior-tile kernel takes two thirds, the edge-tile kernel the
// rest (part[] holds two sums per CTA of both)
int residual_fx_blocks(int num_sms);
// r = oscale (fhat - (B kron I + kappa I kron A) u) in FP32 for the bidiagonal B with
// nonzeros at (k,k) and (k, k+off mod n); kbd[k] = (bd_k, bs_k), ku0[k] = u0coef_k and ihf =
// kappa/h^2 as float-float pairs; part[2b], part[2b+1] = per-CTA sums of |oscale r|^2 and
// (want_f) |fscale fhat|^2 over residual_fx_blocks() CTAs; fc_out/fc_in: fhat cache
void launch_residual_fx(cudaStream_t s, int blocks, int N, int n, int off, float2 ihf, float *r,
                        const double *u, const double *f, const double *u0, const float4 *kbd,
                        const float2 *ku0, float oscale, float fscale, bool want_f, double *part,
                        const float2 *fc_in, float2 *fc_out);

// ---- FP64 refinement of the shifted systems (shift_refine.cu) ----
// CTAs per shift of the shifted residuals (gx): one wave of two CTAs per SM over all shifts
int shift_residual_blocks(int N, int n, int num_sms);
// the same residual without FP64 instructions (residual_ws.cu); z must not be NULL and
// the sums of |b|^2 are not formed; sc[j]: per-shift power-of-two scale of the output
void launch_shift_residual_fx(cudaStream_t s, int gx, int N, int n, const double2 *z, const double2 *b,
                              const double2 *lam, double off, float oscale, const float *sc, View out,
                              const int *frozen, double *part);
void launch_round_to_float(cudaStream_t s, long long count, const double *x, float *y);
// dst = src for n16 16-byte words (both 16-byte aligned), streaming loads and stores
void launch_stream_copy(cudaStream_t s, int blocks, const void *src, void *dst, long long n16);
void launch_shift_residual(cudaStream_t s, int gx, int N, int n, const double2 *z, const double2 *b,
                           const double2 *c1, double off, float oscale, const float *sc, View out,
                           const int *frozen, bool want_b, double *part);
void launch_shift_update(cudaStream_t s, int N, int n, double2 *z, View z0, View z1,
                         const int *final_buf, const int *frozen, const float *sc, bool accumulate);

struct CoarsePlan {
  int lc;                   // first level handled inside one CTA per shift
  int L;                    // total levels
  int Ns[kMaxLevels];       // interior sizes per level
  int gamma, nu1, nu2;
  int jacobi;
};
template <typename T> struct CoarseArgs {
  CoarsePlan plan;
  int n;
  int start;   // level the launch starts at
  int block0;  // first CTA of these shifts in the launch (shift j runs in CTA block0 + j)
  const Coef<T> *coef;
  const typename Cx<T>::type *cinv;
};
// one instance's coarse levels in a batched launch (k_coarse_multi)
template <typename T> struct CoarseTask {
  CoarseArgs<T> a;
  View b, z;  // bt and z of the first coarse level
  const int *active;
};
template <typename T>
size_t coarse_smem_bytes(const CoarsePlan &plan, int start);
template <typename T>
cudaError_t prepare_coarse(size_t smem);
// Levels start..L-1 in one CTA per shift; see k_coarse for the two modes.
template <typename T>
void launch_coarse(cudaStream_t s, const CoarsePlan &plan, int start, int n, View b, T bscale,
                   View z, const Coef<T> *coef /*[L][n]*/, const typename Cx<T>::type *cinv,
                   const int *active, int ncycles, int load_z, int solve_mode, double tol,
                   int maxit, SolveState st);
// batched launches over several instances (tasks in device memory): the coarse levels
// (ncycles cycles from z = 0, CTAs = total shifts), the convergence test and the end of a
// solve without a final residual (batch_nactive: the count of active shifts of all tasks)
template <typename T>
void launch_coarse_multi(cudaStream_t s, const CoarseTask<T> *tasks, int ntasks, int blocks, size_t smem,
                         int ncycles);
struct ConvTask {
  SolveState st;
  int n, ntiles, j0;  // shifts, norm partials per shift, first global shift index
};
void launch_converge_multi(cudaStream_t s, const ConvTask *tasks, int ntasks, int total, double tol,
                           int maxit, double stall, int cur_buf, int *batch_nactive);
void launch_finalize_multi(cudaStream_t s, const ConvTask *tasks, int ntasks, int total, int cur_buf,
                           int *batch_nactive);
template <typename T>
void launch_copy_scale(cudaStream_t s, int N, int n, View dst, View src, T scale);
template <typename T>
void launch_gather_final(cudaStream_t s, int N, int n, View dst, View z0, View z1,
                         const int *final_buf);

// ---- fused TMA kernels (fused_kernels.cu) ----
struct FusedGeom {
  int TX, TY;                 // output tile (columns, rows)
  int sr_zw, sr_zh, sr_bw, sr_bh;                 // smooth+restrict boxes (complex elements)
  int ps_zw, ps_zh, ps_ew, ps_eh, ps_bw, ps_bh;   // prolong+smooth boxes
};
template <typename T> FusedGeom fused_geom();
template <typename T> cudaError_t prepare_fused();
int fused_tiles(int N, int TX, int TY);
template <typename T>
void launch_smooth_restrict(cudaStream_t s, int grid, const CUtensorMap &zmap,
                            const CUtensorMap &bmap, int N, int n, View zout, View bc,
                            const Coef<T> *coef, const int *active, bool z_zero, double *partials,
                            int part_stride, int *errflag);
template <typename T>
void launch_prolong_smooth(cudaStream_t s, int grid, const CUtensorMap &zmap,
                           const CUtensorMap &emap, const CUtensorMap &bmap, int N, int n,
                           View zout, const Coef<T> *coef, const int *active, int *errflag);

// ---- warp-streaming fused kernels (stream_kernels.cu) ----
// one instance-level of a batched launch: units ubegin .. ubegin + n stream_units(N, seg)
// of the launch; x = the coarse RHS bt_c (smoothing + restriction) or the coarse
// correction e (interpolation + smoothing); partials (smoothing + restriction of a finest
// level only) receive the per-unit |rt|^2 sums
template <typename T> struct StreamTask {
  int N, n, seg, ubegin;
  View z, b, zout, x;
  const Coef<T> *coef;
  const int *active;
  double *partials;
  int part_stride;
};
template <typename T>
void launch_sr_multi(cudaStream_t s, int grid, const StreamTask<T> *tasks, int ntasks, int total, bool z_zero,
                     bool norm);
template <typename T>
void launch_ps_multi(cudaStream_t s, int grid, const StreamTask<T> *tasks, int ntasks, int total);
// work units (strips x segments of `seg` rows) per shift = norm partials per shift
int stream_units(int N, int seg);
template <typename T> int stream_grid(int num_sms);
template <typename T> cudaError_t prepare_stream();
template <typename T>
void launch_sr_stream(cudaStream_t s, int grid, int N, int n, int seg, View z, View b, View zout,
                      View bc, const Coef<T> *coef, const int *active, bool z_zero, double *partials,
                      int part_stride);
template <typename T>
void launch_ps_stream(cudaStream_t s, int grid, int N, int n, int seg, View z, View e, View b,
                      View zout, const Coef<T> *coef, const int *active);

// ---- transforms (transforms.cu) ----
template <typename T>
cudaError_t prepare_transforms(int n);
// g (view, working type) = scale * W fhat, fhat_k = f_k + u0coef[k] u0 (f, u0 double)
template <typename T>
void launch_transform_forward(cudaStream_t s, int N, int n, View g, const void *f, bool f32,
                              const double *u0, const double *u0coef,
                              const typename Cx<T>::type *W, double scale);
// u (double, [n][N][N]) = or += Re(W z); z_j read from z1 where final_buf[j] != 0
// (final_buf may be NULL: all from z0); imag_check: atomicMax of max|Im| bits
template <typename T>
void launch_transform_inverse(cudaStream_t s, int N, int n, double *u, View z0, View z1,
                              const int *final_buf, const typename Cx<T>::type *W, T dscale,
                              bool accumulate, bool imag_check, unsigned long long *imag_max_bits);
// r = fhat - (B kron I + I kron A) u in FP64 (r may be NULL); part[2b], part[2b+1] =
// per-CTA sums of r^2 and fhat^2 over allatonce_blocks() CTAs
int allatonce_blocks();
void launch_allatonce_residual(cudaStream_t s, int N, int n, double kappa, double *r, const double *u,
                               const double *f, const double *u0, const double *u0coef,
                               const int *Bptr, const int *Bcol, const double *Bval,
                               double *part);

// r = fhat - (B kron I + kappa I kron A) u for B with nonzeros only at (k,k) (bd) and
// (k, k+off mod n) (bs), off = -1 or +1; r written as FP64 (r64) or FP32 (r32, times the
// power of two oscale, its sums those of the scaled values), or not at all; part as above,
// the fhat sums only when want_f
void launch_residual_bidiag(cudaStream_t s, int N, int n, int off, double kappa, double *r64,
                            float *r32, const double *u, const double *f, const double *u0,
                            const double *u0coef, const double *bd, const double *bs, bool want_f,
                            double *part, double oscale = 1.0);

// gu0 = sum_k u0coef[k] w_k
void launch_initial_value_gradient(cudaStream_t s, int N, int n, const double *w,
                                   const double *u0coef, double *gu0);
// part[2b] = per-CTA sums of w . (A u) over allatonce_blocks() CTAs (FP64)
void launch_laplacian_dot(cudaStream_t s, int N, int n, const double *w, const double *u,
                          double *part);

// ---- tensor-core transforms (tc_transforms.cu), FP32 working type, n <= 128 ----
bool tc_transforms_supported(int N, int n);
cudaError_t prepare_tc_transforms();
cudaError_t tc_launch_grid(int num_sms, int n, bool inverse, int *grid);
// floats of one split of the forward (inverse = false) or inverse operand for n shifts
size_t tc_operand_floats(int n, bool inverse);
void tc_build_operands(int n, const double *Vinv, const double *V, double scale, float *fwd_hi,
                       float *fwd_lo, float *inv_hi, float *inv_lo);
void launch_tc_forward(cudaStream_t s, int grid, int N, int n, View g, const void *f, bool f32,
                       const double *u0, const double *u0coef, const float *Ahi, const float *Alo,
                       double in_scale, int *errflag);
void launch_tc_inverse(cudaStream_t s, int grid, int N, int n, double *u, View z0, View z1,
                       const int *final_buf, const float *Ahi, const float *Alo, float dscale,
                       bool accumulate, bool imag_check, unsigned long long *imag_bits, int *errflag);

// ---- host-side setup (setup.cpp) ----
void vanka_abc(double er, double ei, double out[6]);
double lfa_omega_opt(double er, double ei, int jacobi);
int invert_dense(int m, std::vector<double> &A /* 2*m*m, complex row-major */);
// B = V D V^{-1} of the real n x n row-major B (eig.cpp): lam 2n doubles, V and Vinv
// 2*n*n doubles (complex interleaved, row-major, columns of V of unit 2-norm).  Returns 0,
// or a negative code (non-finite B, no convergence, a zero eigenvector, singular V).
int diagonalize(int n, const double *B, std::vector<double> &lam, std::vector<double> &V,
                std::vector<double> &Vinv);

}  // namespace pd
