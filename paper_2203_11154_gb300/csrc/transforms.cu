// Time-direction transforms of eq. (1), (V^{-1} kron I_h) and (V kron I_h), applied to
// every grid point, and the FP64 residual of the all-at-once system (1).
//
// Layout: time/shift index outermost, [n][N][N]; one CTA owns kPts consecutive grid
// points, stages their n values in shared memory and forms all n outputs for them.
#include "cplx.cuh"
#include "pd_internal.h"

#include <algorithm>

namespace pd {

namespace {

constexpr int kPts = 32, kGroups = 4, kThreads = kPts * kGroups;

template <typename C>
__device__ __forceinline__ C ldv(const View &v, int j, long long i, long long c) {
  return reinterpret_cast<const C *>(v.p)[j * v.plane + i * v.pitch + c];
}
template <typename C>
__device__ __forceinline__ void stv(const View &v, int j, long long i, long long c, C x) {
  reinterpret_cast<C *>(v.p)[j * v.plane + i * v.pitch + c] = x;
}

// g_j = scale * sum_k W[j][k] fhat_k, fhat_k = f_k + u0coef[k] u0 (real input).
template <typename T, typename InT>
__global__ void __launch_bounds__(kThreads)
k_transform_forward(int N, int n, View g, const InT *__restrict__ f,
                    const double *__restrict__ u0, const double *__restrict__ u0coef,
                    const typename Cx<T>::type *__restrict__ W, T scale) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);  // [n][kPts]
  const long long m = (long long)N * N;
  const long long x0 = (long long)blockIdx.x * kPts;
  for (int t = threadIdx.x; t < n * kPts; t += kThreads) {
    const int k = t / kPts, p = t - k * kPts;
    const long long x = x0 + p;
    double v = 0.0;
    if (x < m) {
      v = (double)f[k * m + x];
      if (u0) v += u0coef[k] * u0[x];
    }
    xs[t] = (T)v;
  }
  __syncthreads();
  const int p = threadIdx.x % kPts, jg = threadIdx.x / kPts;
  const long long x = x0 + p;
  if (x >= m) return;
  const int i = (int)(x / N), c = (int)(x - (long long)i * N);
  for (int j = jg; j < n; j += kGroups) {
    const C *w = W + (long long)j * n;
    T re = 0, im = 0;
    for (int k = 0; k < n; k++) {
      const C wk = w[k];
      const T xv = xs[k * kPts + p];
      re = fmadd(wk.x, xv, re);
      im = fmadd(wk.y, xv, im);
    }
    stv<C>(g, j, i, c, cx<C>(re * scale, im * scale));
  }
}

// u_k (+)= dscale Re sum_j W[k][j] z_j; with imag_check also max |dscale Im sum_j W[k][j] z_j|.
// z_j is read from z1 where final_buf[j] is set, else from z0.  dscale is a power of two.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_transform_inverse(int N, int n, double *__restrict__ u, View z0, View z1,
                    const int *__restrict__ final_buf, const typename Cx<T>::type *__restrict__ W,
                    T dscale, int accumulate, int imag_check, unsigned long long *imag_bits) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *zs = reinterpret_cast<C *>(smem_raw);  // [n][kPts]
  __shared__ double red[kThreads / 32];
  const long long m = (long long)N * N;
  const long long x0 = (long long)blockIdx.x * kPts;
  for (int t = threadIdx.x; t < n * kPts; t += kThreads) {
    const int j = t / kPts, p = t - j * kPts;
    const long long x = x0 + p;
    C v = czero<C>();
    if (x < m) {
      const int i = (int)(x / N), c = (int)(x - (long long)i * N);
      v = (final_buf && final_buf[j]) ? ldv<C>(z1, j, i, c) : ldv<C>(z0, j, i, c);
    }
    zs[t] = v;
  }
  __syncthreads();
  const int p = threadIdx.x % kPts, kg = threadIdx.x / kPts;
  const long long x = x0 + p;
  double imax = 0.0;
  if (x < m) {
    for (int k = kg; k < n; k += kGroups) {
      const C *w = W + (long long)k * n;
      T re = 0, im = 0;
      for (int j = 0; j < n; j++) {
        const C wj = w[j];
        const C zv = zs[j * kPts + p];
        re = fmadd(wj.x, zv.x, re);
        re = fmadd(-wj.y, zv.y, re);
        if (imag_check) {
          im = fmadd(wj.x, zv.y, im);
          im = fmadd(wj.y, zv.x, im);
        }
      }
      double out = (double)(re * dscale);
      if (accumulate) out += u[k * m + x];
      u[k * m + x] = out;
      imax = fmax(imax, fabs((double)(im * dscale)));
    }
  }
  if (imag_check) {
    for (int o = 16; o > 0; o >>= 1) imax = fmax(imax, __shfl_down_sync(0xffffffffu, imax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = imax;
    __syncthreads();
    if (threadIdx.x == 0) {
      double mx = 0.0;
      for (int k = 0; k < kThreads / 32; k++) mx = fmax(mx, red[k]);
      atomicMax(imag_bits, (unsigned long long)__double_as_longlong(mx));
    }
  }
}

constexpr int kResThreads = 256;

// r_k = fhat_k - sum_l B[k][l] u_l - kappa A u_k (eq. (1)), A = (1/h^2) 5-point, FP64.
// part[2b], part[2b+1]: this CTA's sums of r^2 and fhat^2 (fixed grid, fixed order).
__global__ void __launch_bounds__(kResThreads)
k_allatonce_residual(int N, int n, double *__restrict__ r, const double *__restrict__ u,
                     const double *__restrict__ f, const double *__restrict__ u0,
                     const double *__restrict__ u0coef, const int *__restrict__ Bptr,
                     const int *__restrict__ Bcol, const double *__restrict__ Bval, double ih2,
                     double *__restrict__ part) {
  __shared__ double red[2][kResThreads / 32];
  const long long m = (long long)N * N, total = m * n;
  double ar = 0.0, af = 0.0;
  for (long long q = (long long)blockIdx.x * kResThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kResThreads) {
    const int k = (int)(q / m);
    const long long x = q - (long long)k * m;
    const int i = (int)(x / N), c = (int)(x - (long long)i * N);
    double fh = f[q];
    if (u0) fh += u0coef[k] * u0[x];
    double bu = 0.0;
    for (int e = Bptr[k]; e < Bptr[k + 1]; e++) bu += Bval[e] * u[(long long)Bcol[e] * m + x];
    const double *uk = u + (long long)k * m;
    double nb = 0.0;
    if (i > 0) nb += uk[x - N];
    if (i < N - 1) nb += uk[x + N];
    if (c > 0) nb += uk[x - 1];
    if (c < N - 1) nb += uk[x + 1];
    const double rv = fh - bu - ih2 * (4.0 * uk[x] - nb);
    if (r) r[q] = rv;
    ar += rv * rv;
    af += fh * fh;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, o);
    af += __shfl_down_sync(0xffffffffu, af, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ar;
    red[1][threadIdx.x >> 5] = af;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kResThreads / 32; w++) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

// Residual of eq. (1) for a B with nonzeros only at (k, k) and (k, k+off mod n), off = -1
// (backward Euler, its alpha-circulant variant) or +1 (their transposes, the adjoint):
//   r_k = fhat_k - (bd_k u_k + bs_k u_{k+off mod n}) - (kappa/h^2)(4 u_k - sum of 4 neighbours)
// with 6 FP64 operations per point (GB300's FP64 rate bounds this kernel).  One CTA
// sweeps whole grid rows (k, i); per-CTA sums of r^2 (and of fhat^2 when WANT_F) go to
// part[2b], part[2b+1] over a fixed grid, so the sums are reproducible.
template <typename OutT, bool WANT_F>
__global__ void __launch_bounds__(kResThreads)
k_residual_bidiag(int N, int n, int off, OutT *__restrict__ r, const double *__restrict__ u,
                  const double *__restrict__ f, const double *__restrict__ u0,
                  const double *__restrict__ u0coef, const double *__restrict__ bd,
                  const double *__restrict__ bs, double ih2, double oscale, double *__restrict__ part) {
  __shared__ double red[2][kResThreads / 32];
  const long long m = (long long)N * N;
  double ar = 0.0, af = 0.0;
  for (int row = blockIdx.x; row < n * N; row += gridDim.x) {
    const int k = row / N, i = row - k * N;
    const int kp = (k + off + n) % n;
    // r = fhat - (bd + 4 kappa/h^2) u - bs u_prev + (kappa/h^2)(sum of neighbours):
    // 3 additions and 3 FMAs in FP64 per point; with an FP32 output (the refinement's
    // residual, whose norm only decides when to stop) |r|^2 of a row is summed in FP32
    // and added to the FP64 total per row, else in FP64
    const double c1 = bd[k] + 4.0 * ih2, sk = bs[k], ck = u0 ? u0coef[k] : 0.0;
    const double *uk = u + (long long)k * m + (long long)i * N;
    const double *up = u + (long long)kp * m + (long long)i * N;
    const double *fk = f + (long long)k * m + (long long)i * N;
    const double *u0r = u0 ? u0 + (long long)i * N : nullptr;
    float arow = 0.f;
    double arow64 = 0.0;
    for (int c = threadIdx.x; c < N; c += kResThreads) {
      double fh = fk[c];
      if (ck != 0.0) fh = fma(ck, u0r[c], fh);
      double nb = (c > 0 ? uk[c - 1] : 0.0) + (c < N - 1 ? uk[c + 1] : 0.0);
      if (i > 0) nb += uk[c - N];
      if (i < N - 1) nb += uk[c + N];
      const double rv = fma(ih2, nb, fma(-sk, up[c], fma(-c1, uk[c], fh)));
      if (sizeof(OutT) == 4) {
        // the FP32 output times the power of two oscale (kept near unit size)
        const float rf = (float)(rv * oscale);
        if (r) r[(long long)k * m + (long long)i * N + c] = (OutT)rf;
        arow = fmaf(rf, rf, arow);
      } else {
        if (r) r[(long long)k * m + (long long)i * N + c] = (OutT)rv;
        arow64 = fma(rv, rv, arow64);
      }
      if (WANT_F) af = fma(fh, fh, af);
    }
    ar += (double)arow + arow64;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, o);
    if (WANT_F) af += __shfl_down_sync(0xffffffffu, af, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ar;
    red[1][threadIdx.x >> 5] = af;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kResThreads / 32; w++) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

// sum over k, x of w_k(x) (A u_k)(x), A = (1/h^2) 5-point, FP64, per-CTA partials
__global__ void __launch_bounds__(kResThreads)
k_laplacian_dot(int N, int n, const double *__restrict__ w, const double *__restrict__ u,
                double ih2, double *__restrict__ part) {
  __shared__ double red[kResThreads / 32];
  const long long m = (long long)N * N;
  double acc = 0.0;
  for (int row = blockIdx.x; row < n * N; row += gridDim.x) {
    const int k = row / N, i = row - k * N;
    const double *uk = u + (long long)k * m + (long long)i * N;
    const double *wk = w + (long long)k * m + (long long)i * N;
    for (int c = threadIdx.x; c < N; c += kResThreads) {
      double nb = 0.0;
      if (i > 0) nb += uk[c - N];
      if (i < N - 1) nb += uk[c + N];
      if (c > 0) nb += uk[c - 1];
      if (c < N - 1) nb += uk[c + 1];
      acc = fma(wk[c], ih2 * fma(4.0, uk[c], -nb), acc);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0;
    for (int q = 0; q < kResThreads / 32; q++) s0 += red[q];
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// gu0 = sum_k u0coef[k] w_k (FP64): the gradient with respect to the initial value
__global__ void k_initial_value_gradient(long long m, int n, const double *__restrict__ w,
                                         const double *__restrict__ u0coef, double *__restrict__ gu0) {
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < m;
       x += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n; k++)
      if (u0coef[k] != 0.0) s = fma(u0coef[k], w[(long long)k * m + x], s);
    gu0[x] = s;
  }
}

}  // namespace

void launch_initial_value_gradient(cudaStream_t s, int N, int n, const double *w,
                                   const double *u0coef, double *gu0) {
  const long long m = (long long)N * N;
  k_initial_value_gradient<<<(unsigned)std::min<long long>((m + 255) / 256, 4096), 256, 0, s>>>(
      m, n, w, u0coef, gu0);
}

void launch_laplacian_dot(cudaStream_t s, int N, int n, const double *w, const double *u,
                          double *part) {
  const double h = 1.0 / (N + 1);
  k_laplacian_dot<<<allatonce_blocks(), kResThreads, 0, s>>>(N, n, w, u, 1.0 / (h * h), part);
}

void launch_residual_bidiag(cudaStream_t s, int N, int n, int off, double kappa, double *r64,
                            float *r32, const double *u, const double *f, const double *u0,
                            const double *u0coef, const double *bd, const double *bs, bool want_f,
                            double *part, double oscale) {
  const double h = 1.0 / (N + 1), ih2 = kappa / (h * h);
  const int g = allatonce_blocks();
  if (r32) {
    if (want_f)
      k_residual_bidiag<float, true><<<g, kResThreads, 0, s>>>(N, n, off, r32, u, f, u0, u0coef, bd, bs, ih2, oscale, part);
    else
      k_residual_bidiag<float, false><<<g, kResThreads, 0, s>>>(N, n, off, r32, u, f, u0, u0coef, bd, bs, ih2, oscale, part);
  } else {
    if (want_f)
      k_residual_bidiag<double, true><<<g, kResThreads, 0, s>>>(N, n, off, r64, u, f, u0, u0coef, bd, bs, ih2, oscale, part);
    else
      k_residual_bidiag<double, false><<<g, kResThreads, 0, s>>>(N, n, off, r64, u, f, u0, u0coef, bd, bs, ih2, oscale, part);
  }
}

template <typename T>
cudaError_t prepare_transforms(int n) {
  using C = typename Cx<T>::type;
  cudaError_t e = cudaFuncSetAttribute(k_transform_forward<T, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(n * kPts * sizeof(T)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_transform_forward<T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(n * kPts * sizeof(T)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_transform_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(n * kPts * sizeof(C)));
}

template <typename T>
void launch_transform_forward(cudaStream_t s, int N, int n, View g, const void *f, bool f32,
                              const double *u0, const double *u0coef,
                              const typename Cx<T>::type *W, double scale) {
  const long long m = (long long)N * N;
  const unsigned blocks = (unsigned)((m + kPts - 1) / kPts);
  if (f32)
    k_transform_forward<T, float><<<blocks, kThreads, n * kPts * sizeof(T), s>>>(
        N, n, g, static_cast<const float *>(f), u0, u0coef, W, (T)scale);
  else
    k_transform_forward<T, double><<<blocks, kThreads, n * kPts * sizeof(T), s>>>(
        N, n, g, static_cast<const double *>(f), u0, u0coef, W, (T)scale);
}

template <typename T>
void launch_transform_inverse(cudaStream_t s, int N, int n, double *u, View z0, View z1,
                              const int *final_buf, const typename Cx<T>::type *W, T dscale,
                              bool accumulate, bool imag_check,
                              unsigned long long *imag_max_bits) {
  using C = typename Cx<T>::type;
  const long long m = (long long)N * N;
  const unsigned blocks = (unsigned)((m + kPts - 1) / kPts);
  k_transform_inverse<T><<<blocks, kThreads, n * kPts * sizeof(C), s>>>(
      N, n, u, z0, z1, final_buf, W, dscale, accumulate ? 1 : 0, imag_check ? 1 : 0, imag_max_bits);
}

int allatonce_blocks() { return 4 * 152; }

void launch_allatonce_residual(cudaStream_t s, int N, int n, double kappa, double *r, const double *u,
                               const double *f, const double *u0, const double *u0coef,
                               const int *Bptr, const int *Bcol, const double *Bval,
                               double *part) {
  const double h = 1.0 / (N + 1);
  k_allatonce_residual<<<allatonce_blocks(), kResThreads, 0, s>>>(
      N, n, r, u, f, u0, u0coef, Bptr, Bcol, Bval, kappa / (h * h), part);
}

template cudaError_t prepare_transforms<double>(int);
template cudaError_t prepare_transforms<float>(int);
template void launch_transform_forward<double>(cudaStream_t, int, int, View, const void *, bool,
                                               const double *, const double *, const double2 *,
                                               double);
template void launch_transform_forward<float>(cudaStream_t, int, int, View, const void *, bool,
                                              const double *, const double *, const float2 *,
                                              double);
template void launch_transform_inverse<double>(cudaStream_t, int, int, double *, View, View,
                                               const int *, const double2 *, double, bool, bool,
                                               unsigned long long *);
template void launch_transform_inverse<float>(cudaStream_t, int, int, double *, View, View,
                                              const int *, const float2 *, float, bool, bool,
                                              unsigned long long *);

}  // namespace pd
