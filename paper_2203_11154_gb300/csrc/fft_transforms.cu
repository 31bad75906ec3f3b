// Time transforms of eq. (1) for the alpha-circulant backward-Euler B by FFT.
//
// With B = (1/tau)(I - C_alpha) the eigenvector matrices are scaled Fourier matrices:
//   V^{-1}[j][k] = alpha^{k/n} e^{+2 pi i j k / n} / n,   V[k][j] = alpha^{-k/n} e^{-2 pi i k j / n},
// so at every grid point
//   forward:  g_j = s/n sum_k e^{+2 pi i j k / n} (alpha^{k/n} fhat_k)       (s = h^2/kappa or 1)
//   inverse:  u_k (+)= alpha^{-k/n} Re sum_j e^{-2 pi i k j / n} z_j
// are a weighted DFT of length n, O(n log n) per point instead of the O(n^2) dense product.
//
// TP threads (1, 2 or 4, see fft_tp) per grid point, P points per CTA.  n = N1 N2 (both
// powers of two): the four-step decomposition
//   X[k1 + N1 k2] = sum_{j2} w_n^{j2 k1} [sum_{j1} x[N2 j1 + j2] w_{N1}^{j1 k1}] w_{N2}^{j2 k2}
// with the small DFTs as unrolled radix-2 butterflies in registers and the n values of a
// point in its own column of shared memory ([n][P], conflict-free); the TP threads of a
// point share the small DFTs of each pass, with CTA barriers around the passes.  Loads
// and stores of the n time slices are coalesced across the threads of a warp (consecutive
// grid points).
#include <algorithm>

#include "cplx.cuh"
#include "fpbits.cuh"
#include "pd_internal.h"
#include "tma.cuh"

namespace pd {
namespace {

// grid points (threads) per CTA: up to 128, with the CTA's columns within 96 KB of shared
// memory (a multiple of 32)
template <typename T, int n> __host__ __device__ constexpr int fft_points() {
  return (98304 / (n * (int)sizeof(typename Cx<T>::type))) >= 128
             ? 128
             : ((98304 / (n * (int)sizeof(typename Cx<T>::type))) / 32) * 32;
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; b++) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

// in-place DFT of length R (power of two) of v in registers: v_out[k] = sum_j v[j] w^{jk},
// w = tw[step] (tw[t] = w_n^t, n = R * step), radix-2 decimation in time
// one radix-2 stage of span M (butterflies (k + j, k + j + M/2), twiddle w^{j R/M}),
// then the next stage; the stages are a compile-time recursion so that every index is a
// constant and v stays in registers
template <typename C, int R, int M>
__device__ __forceinline__ void dft_stages(C (&v)[R], const C *__restrict__ tw, int step) {
  if constexpr (M <= R) {
#pragma unroll
    for (int k = 0; k < R; k += M) {
#pragma unroll
      for (int j = 0; j < M / 2; j++) {
        C t = v[k + j + M / 2];
        if (j != 0) t = cmul(tw[j * (R / M) * step], t);
        v[k + j + M / 2] = csub(v[k + j], t);
        v[k + j] = cadd(v[k + j], t);
      }
    }
    dft_stages<C, R, 2 * M>(v, tw, step);
  }
}

template <typename C, int R>
__device__ __forceinline__ void dft_small(C (&v)[R], const C *__restrict__ tw, int step) {
  constexpr int bits = ilog2(R);
#pragma unroll
  for (int i = 0; i < R; i++) {
    const int r = bitrev(i, bits);
    if (r > i) {
      const C t = v[i];
      v[i] = v[r];
      v[r] = t;
    }
  }
  dft_stages<C, R, 2>(v, tw, step);
}

// the two passes of the four-step DFT on the point's column col[e * P], shared by the TP
// threads of the point (thread t takes every TP-th small DFT of each pass); the CTA
// synchronises before and between the passes
template <typename C, int N1, int N2, int P, int TP>
__device__ __forceinline__ void fft_column(C *col, const C *__restrict__ tw, int t) {
  constexpr int n = N1 * N2;
  __syncthreads();
  // pass 1: for each j2, DFT over j1 of x[N2 j1 + j2], times w_n^{j2 k1}
  for (int j2 = t; j2 < N2; j2 += TP) {
    C v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; j1++) v[j1] = col[(N2 * j1 + j2) * P];
    dft_small<C, N1>(v, tw, N2);
#pragma unroll
    for (int k1 = 0; k1 < N1; k1++) {
      const C x = (k1 == 0 || j2 == 0) ? v[k1] : cmul(tw[(j2 * k1) % n], v[k1]);
      col[(N2 * k1 + j2) * P] = x;
    }
  }
  __syncthreads();
  // pass 2: for each k1, DFT over j2; X[k1 + N1 k2] ends in slot N2 k1 + k2
  for (int k1 = t; k1 < N1; k1 += TP) {
    C v[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; j2++) v[j2] = col[(N2 * k1 + j2) * P];
    dft_small<C, N2>(v, tw, N1);
#pragma unroll
    for (int k2 = 0; k2 < N2; k2++) col[(N2 * k1 + k2) * P] = v[k2];
  }
  __syncthreads();
}

// threads per grid point: four for n = 128 (both passes have at least eight small DFTs
// there) and for the inverse at n = 64 (measured: inverse 3 % faster, forward 3 % slower
// than with two), two where both passes have at least two, else one
template <int N1, int N2, bool INV> __host__ __device__ constexpr int fft_tp() {
  return (N1 >= 4 && N2 >= 4 && (N1 * N2 >= 128 || (INV && N1 * N2 >= 64)))
             ? 4
             : ((N1 >= 2 && N2 >= 2) ? 2 : 1);
}
// CTAs per SM that the shared memory allows, at most 3 and at most 1024 threads (64
// registers a thread at least), for the register budget
template <typename T, int N1, int N2, bool INV> __host__ __device__ constexpr int fft_min_blocks() {
  constexpr int n = N1 * N2, th = fft_points<T, n>() * fft_tp<N1, N2, INV>();
  constexpr int by_smem = 229376 / (n * fft_points<T, n>() * (int)sizeof(typename Cx<T>::type));
  constexpr int a = by_smem < 3 ? by_smem : 3, b = 1024 / th;
  return (a < b ? a : b) < 1 ? 1 : (a < b ? a : b);
}

__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

// an input value as the transform's type: FP64 into FP32 by bits, otherwise as is
template <typename T, typename InT> __device__ __forceinline__ T as_t(InT v) {
  if constexpr (sizeof(T) == 4 && sizeof(InT) == 8) return f64_to_f32(v);
  else return (T)v;
}

template <typename T, typename InT> __device__ __forceinline__ T load_in(const InT *p) { return (T)*p; }

// g_j(point) = wk-weighted DFT (+ exponent) of fhat; wk[k] = s alpha^{k/n} / n.  Thread
// (t, p) of the CTA (p = threadIdx.x % P) serves point p: its loads and stores are the time
// slices t, t + TP, ..., so a warp touches 32 consecutive points of one slice.  With FP32
// input at most two CTAs a SM: the registers hold a thread's slices (see below).
template <typename T, int N1, int N2, typename InT>
__global__ void __launch_bounds__(fft_points<T, N1 * N2>() * fft_tp<N1, N2, false>(),
                                  (sizeof(InT) == 4 && fft_min_blocks<T, N1, N2, false>() > 2)
                                      ? 2
                                      : fft_min_blocks<T, N1, N2, false>())
k_fft_forward(int N, View g, const InT *__restrict__ f, const double *__restrict__ u0,
              const double *__restrict__ u0coef, const T *__restrict__ wk,
              const typename Cx<T>::type *__restrict__ tw) {
  using C = typename Cx<T>::type;
  constexpr int n = N1 * N2, P = fft_points<T, n>(), TP = fft_tp<N1, N2, false>();
  extern __shared__ __align__(16) unsigned char fft_raw[];
  const int p = threadIdx.x % P, t = threadIdx.x / P;
  C *col = reinterpret_cast<C *>(fft_raw) + p;
  const long long m = (long long)N * N;
  constexpr int kPer = n / TP;                         // slices per thread
  // loads in flight per thread: all of an FP32 input when there are 32 (measured 5 %
  // faster at n = 64 than 16), else up to 16
  constexpr int kBatch = (sizeof(InT) == 4 && kPer >= 32) ? 32 : (kPer < 16 ? kPer : 16);
  for (long long base = (long long)blockIdx.x * P; base < m; base += (long long)gridDim.x * P) {
    const long long x = base + p;
    const bool ok = x < m;
    const double u0x = (ok && u0) ? u0[x] : 0.0;
    if constexpr (kBatch == kPer && sizeof(InT) == 4) {
      // The thread's slices k = TP q + t are exactly the inputs of its pass-1 DFTs
      // (j2 = t + TP r takes x[N2 j1 + j2], i.e. q = (N2/TP) j1 + r), so they go from
      // registers into pass 1, and pass 2 writes its outputs straight to g: one exchange
      // through the shared-memory column and two barriers per tile.
      InT in[kPer];
#pragma unroll
      for (int q = 0; q < kPer; q++) in[q] = ok ? f[(long long)(TP * q + t) * m + x] : (InT)0;
      constexpr int R1 = N2 / TP;
#pragma unroll
      for (int r = 0; r < R1; r++) {
        const int j2 = t + TP * r;
        C v[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; j1++) {
          const int q = R1 * j1 + r, k = TP * q + t;
          const double ck = u0 ? u0coef[k] : 0.0;
          T val;
          if (u0 && (__double_as_longlong(ck) << 1) != 0) val = (T)(to_f64(in[q]) + ck * u0x);
          else val = (T)in[q];
          v[j1] = cx<C>(val * wk[k], (T)0);
        }
        dft_small<C, N1>(v, tw, N2);
#pragma unroll
        for (int k1 = 0; k1 < N1; k1++)
          col[(N2 * k1 + j2) * P] = (k1 == 0 || j2 == 0) ? v[k1] : cmul(tw[(j2 * k1) % n], v[k1]);
      }
      __syncthreads();
      C *gp = nullptr;
      if (ok) {
        const int i = (int)(x / N), c = (int)(x - (long long)i * N);
        gp = reinterpret_cast<C *>(g.p) + (long long)i * g.pitch + c;
      }
      for (int k1 = t; k1 < N1; k1 += TP) {
        C v[N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; j2++) v[j2] = col[(N2 * k1 + j2) * P];
        dft_small<C, N2>(v, tw, N1);
        if (ok) {
#pragma unroll
          for (int k2 = 0; k2 < N2; k2++) gp[(long long)(k1 + N1 * k2) * g.plane] = v[k2];
        }
      }
      __syncthreads();  // the columns are refilled by the next points
      continue;
    }
#pragma unroll 1
    for (int q0 = 0; q0 < kPer; q0 += kBatch) {
      InT in[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; q++)
        in[q] = ok ? f[(long long)(TP * (q0 + q) + t) * m + x] : (InT)0;
#pragma unroll
      for (int q = 0; q < kBatch; q++) {
        const int k = TP * (q0 + q) + t;
        // the initial-value term (FP64) only on the time steps whose coefficient is nonzero
        // (tested on the bits: no FP64 comparison per point)
        const double ck = u0 ? u0coef[k] : 0.0;
        T v;
        if (u0 && (__double_as_longlong(ck) << 1) != 0) v = as_t<T>(to_f64(in[q]) + ck * u0x);
        else v = as_t<T>(in[q]);
        col[k * P] = cx<C>(v * wk[k], (T)0);
      }
    }
    fft_column<C, N1, N2, P, TP>(col, tw, t);
    if (ok) {
      const int i = (int)(x / N), c = (int)(x - (long long)i * N);
      C *gp = reinterpret_cast<C *>(g.p) + (long long)i * g.pitch + c;
#pragma unroll 4
      for (int s = t; s < n; s += TP) {
        const int k1 = s / N2, k2 = s % N2;
        gp[(long long)(k1 + N1 * k2) * g.plane] = col[s * P];
      }
    }
    __syncthreads();  // the columns are refilled by the next points
  }
}

// u_k(point) (+)= dscale wk[k] Re(DFT (- exponent) of z)_k, wk[k] = alpha^{-k/n}, dscale a
// power of two (the inverse of the scale of the FP32 right-hand side); z_j from z1 where
// final_buf[j] is set, else z0; imag_check: atomic max of |dscale wk[k] Im(.)_k| (bits of a
// double)
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(fft_points<T, N1 * N2>() * fft_tp<N1, N2, true>(), fft_min_blocks<T, N1, N2, true>())
k_fft_inverse(int N, double *__restrict__ u, View z0, View z1, const int *__restrict__ final_buf,
              const T *__restrict__ wk, const typename Cx<T>::type *__restrict__ tw, T dscale,
              int accumulate, int imag_check, unsigned long long *imag_bits) {
  using C = typename Cx<T>::type;
  constexpr int n = N1 * N2, P = fft_points<T, n>(), TP = fft_tp<N1, N2, true>();
  extern __shared__ __align__(16) unsigned char fft_raw[];
  __shared__ float red[P * TP / 32];
  const int p = threadIdx.x % P, t = threadIdx.x / P;
  C *col = reinterpret_cast<C *>(fft_raw) + p;
  const long long m = (long long)N * N;
  constexpr int kPer = n / TP;
  constexpr int kBatch = kPer < 16 ? kPer : 16;
  constexpr int kOut = kPer < 8 ? kPer : 8;  // outputs (and accumulated u values) per batch
  float imax = 0.f;
  for (long long base = (long long)blockIdx.x * P; base < m; base += (long long)gridDim.x * P) {
    const long long x = base + p;
    const bool ok = x < m;
    const int i = (int)(x / N), c = (int)(x - (long long)i * N);
    if constexpr (kPer <= 16 && sizeof(T) == 4) {
      // as in k_fft_forward: the thread's slices j = TP q + t are the inputs of its pass-1
      // DFTs, kept in registers; pass 2 writes (or adds) its outputs straight to u
      C in[kPer];
#pragma unroll
      for (int q = 0; q < kPer; q++) {
        const int j = TP * q + t;
        const View &zv = (final_buf && final_buf[j]) ? z1 : z0;
        in[q] = ok ? reinterpret_cast<const C *>(zv.p)[(long long)j * zv.plane + (long long)i * zv.pitch + c]
                   : czero<C>();
      }
      constexpr int R1 = N2 / TP;
#pragma unroll
      for (int r = 0; r < R1; r++) {
        const int j2 = t + TP * r;
        C v[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; j1++) v[j1] = in[R1 * j1 + r];
        dft_small<C, N1>(v, tw, N2);
#pragma unroll
        for (int k1 = 0; k1 < N1; k1++)
          col[(N2 * k1 + j2) * P] = (k1 == 0 || j2 == 0) ? v[k1] : cmul(tw[(j2 * k1) % n], v[k1]);
      }
      __syncthreads();
      for (int k1 = t; k1 < N1; k1 += TP) {
        C v[N2];
#pragma unroll
        for (int j2 = 0; j2 < N2; j2++) v[j2] = col[(N2 * k1 + j2) * P];
        dft_small<C, N2>(v, tw, N1);
        if (ok) {
          constexpr int kO = N2 < 4 ? N2 : 4;  // accumulated u values per batch
#pragma unroll
          for (int k20 = 0; k20 < N2; k20 += kO) {
            double uo[kO];
            if (accumulate) {
#pragma unroll
              for (int q = 0; q < kO; q++) uo[q] = u[(long long)(k1 + N1 * (k20 + q)) * m + x];
            }
#pragma unroll
            for (int q = 0; q < kO; q++) {
              const int k = k1 + N1 * (k20 + q);
              const T wd = wk[k] * dscale;
              const T re = v[k20 + q].x * wd;
              u[(long long)k * m + x] = accumulate ? uo[q] + to_f64(re) : to_f64(re);
              if (imag_check) imax = fmaxf(imax, fabsf((float)(v[k20 + q].y * wd)));
            }
          }
        }
      }
      __syncthreads();  // the columns are refilled by the next points
      continue;
    }
#pragma unroll 1
    for (int q0 = 0; q0 < kPer; q0 += kBatch) {
      C in[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; q++) {
        const int j = TP * (q0 + q) + t;
        const View &zv = (final_buf && final_buf[j]) ? z1 : z0;
        in[q] = ok ? reinterpret_cast<const C *>(zv.p)[(long long)j * zv.plane + (long long)i * zv.pitch + c]
                   : czero<C>();
      }
#pragma unroll
      for (int q = 0; q < kBatch; q++) col[(TP * (q0 + q) + t) * P] = in[q];
    }
    fft_column<C, N1, N2, P, TP>(col, tw, t);
    if (ok) {
#pragma unroll 1
      for (int q0 = 0; q0 < kPer; q0 += kOut) {
        double uo[kOut];
        if (accumulate) {
#pragma unroll
          for (int q = 0; q < kOut; q++) {
            const int s = TP * (q0 + q) + t, k = s / N2 + N1 * (s % N2);
            uo[q] = u[(long long)k * m + x];
          }
        }
#pragma unroll
        for (int q = 0; q < kOut; q++) {
          const int s = TP * (q0 + q) + t, k = s / N2 + N1 * (s % N2);
          const C v = col[s * P];
          const T wd = wk[k] * dscale;
          const T re = v.x * wd;
          u[(long long)k * m + x] = accumulate ? uo[q] + to_f64(re) : to_f64(re);
          if (imag_check) imax = fmaxf(imax, fabsf((float)(v.y * wd)));
        }
      }
    }
    __syncthreads();  // the columns are refilled by the next points
  }
  if (imag_check) {
    for (int o = 16; o > 0; o >>= 1) imax = fmaxf(imax, __shfl_down_sync(0xffffffffu, imax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = imax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float mx = 0.f;
      for (int w = 0; w < P * TP / 32; w++) mx = fmaxf(mx, red[w]);
      atomicMax(imag_bits, (unsigned long long)__double_as_longlong((double)mx));
    }
  }
}

// ---- pipelined FP32 transforms for n = N1 N2 with N2 = 8 (n = 64, 128) ----
//
// Tiles of 32 grid points of one grid row, all n slices.  The CTA's eight warps are the
// N2 = 8 threads of each point (warp t serves the slices t, t + N2, ...: the inputs of its
// pass-1 DFT, j2 = t), the lanes the 32 points.  The input slices of the CTA's next
// kPipeS - 1 tiles are in flight in a cp.async ring of shared-memory stages while the
// current tile is transformed: pass 1 reads its slices from the stage, pass 2 (N1 / N2
// DFTs of length N2 per thread) reads the exchanged columns and writes to global memory
// directly.  No registers hold prefetched data, so the loads in flight per SM are the
// stages (up to 2 x 64 KB at n = 128), not the registers.
constexpr int kPipeP = 32, kPipeTP = 8, kPipeThreads = kPipeP * kPipeTP, kPipeS = 3;

// g_j(point) = wk-weighted DFT (+ exponent) of fhat at the 32 points of a tile, FP32 work.
// Stage layout [n][32] of the input type; pass 1 writes complex columns into `col`.
template <int N1, typename InT>
__global__ void __launch_bounds__(kPipeThreads)
k_fft_forward_pipe(int N, View g, const InT *__restrict__ f, const double *__restrict__ u0,
                   const double *__restrict__ u0coef, const float *__restrict__ wk,
                   const float2 *__restrict__ tw) {
  constexpr int N2 = kPipeTP, n = N1 * N2, P = kPipeP;
  constexpr int S = sizeof(InT) == 8 ? 2 : kPipeS;  // stages (FP64 input: the first step only)
  extern __shared__ __align__(16) unsigned char fft_raw[];
  InT *stage = reinterpret_cast<InT *>(fft_raw);                     // [S][n][P]
  float2 *col = reinterpret_cast<float2 *>(fft_raw + (size_t)S * n * P * sizeof(InT));  // [n][P]
  const int p = threadIdx.x & 31, t = threadIdx.x >> 5;
  const long long m = (long long)N * N;
  const int tpr = (N + P - 1) / P, total = N * tpr;
  // weights of this thread's slices k = N2 j1 + t, and a bit per slice whose initial-value
  // coefficient is nonzero (tested on the bits: no FP64 comparison)
  float wq[N1];
  unsigned has_u0 = 0;
#pragma unroll
  for (int j1 = 0; j1 < N1; j1++) {
    const int k = N2 * j1 + t;
    wq[j1] = wk[k];
    if (u0 && (__double_as_longlong(u0coef[k]) << 1) != 0) has_u0 |= 1u << j1;
  }
  // copies of one tile: element (k, point q) of the tile, one per thread and step
  auto issue = [&](int tile, int st) {
    if (tile < total) {
      const int i = tile / tpr, c0 = (tile - i * tpr) * P;
      const uint32_t base = smem_u32(stage + (size_t)st * n * P);
#pragma unroll
      for (int e = 0; e < n * P / kPipeThreads; e++) {
        const int q = threadIdx.x + kPipeThreads * e, k = q / P, pt = q % P;
        const bool ok = c0 + pt < N;
        // beyond the grid: zero fill, from the row's last element (a valid address near the
        // data: zero-fill copies still send their source address, and one shared address
        // for all of them would become a hot spot)
        const InT *src = f + (long long)k * m + (long long)i * N + min(c0 + pt, N - 1);
        cpa(base + (uint32_t)(q * sizeof(InT)), src, (int)sizeof(InT), ok);
      }
    }
    cpa_commit();
  };
  int q = 0;
  for (int s0 = 0; s0 < S - 1; s0++) issue(blockIdx.x + s0 * gridDim.x, s0);
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x, q++) {
    issue(tile + (S - 1) * gridDim.x, (q + S - 1) % S);
    cpa_wait<S - 1>();
    __syncthreads();
    const InT *sq = stage + (size_t)(q % S) * n * P;
    const int i = tile / tpr, c = (tile - i * tpr) * P + p;
    const double u0x = (has_u0 && c < N) ? u0[(long long)i * N + c] : 0.0;
    float2 v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; j1++) {
      const InT x = sq[(N2 * j1 + t) * P + p];
      float val;
      if (has_u0 >> j1 & 1u) val = as_t<float>(to_f64(x) + u0coef[N2 * j1 + t] * u0x);
      else val = as_t<float>(x);
      v[j1] = make_float2(val * wq[j1], 0.f);
    }
    dft_small<float2, N1>(v, tw, N2);
#pragma unroll
    for (int k1 = 0; k1 < N1; k1++)
      col[(N2 * k1 + t) * P + p] = (k1 == 0 || t == 0) ? v[k1] : cmul(tw[(t * k1) % n], v[k1]);
    __syncthreads();
    float2 *gp = reinterpret_cast<float2 *>(g.p) + (long long)i * g.pitch + c;
#pragma unroll
    for (int r = 0; r < N1 / N2; r++) {
      const int k1 = t + N2 * r;
      float2 w[N2];
#pragma unroll
      for (int j2 = 0; j2 < N2; j2++) w[j2] = col[(N2 * k1 + j2) * P + p];
      dft_small<float2, N2>(w, tw, N1);
      if (c < N) {
#pragma unroll
        for (int k2 = 0; k2 < N2; k2++) gp[(long long)(k1 + N1 * k2) * g.plane] = w[k2];
      }
    }
    __syncthreads();  // the stage and the column are refilled next
  }
  cpa_wait<0>();
}

// u_k(point) (+)= dscale wk[k] Re(DFT (- exponent) of z)_k at the 32 points of a tile, FP32
// work.  Stage layout [n][32] complex; pass 1 writes its outputs back into its own slots.
// PAIRS: copies of two points (16 bytes), for z arrays whose pitch and plane are even and
// whose bases are 16-byte aligned (the context's padded levels); else one point (8 bytes).
template <int N1, bool PAIRS>
__global__ void __launch_bounds__(kPipeThreads, N1 <= 8 ? 3 : 2)
k_fft_inverse_pipe(int N, double *__restrict__ u, View z0, View z1, const int *__restrict__ final_buf,
                   const float *__restrict__ wk, const float2 *__restrict__ tw, float dscale,
                   int accumulate, int imag_check, unsigned long long *imag_bits) {
  constexpr int N2 = kPipeTP, n = N1 * N2, P = kPipeP, S = kPipeS;
  constexpr int W = PAIRS ? 2 : 1;                // points per copy
  constexpr int kCh = n * P / W / kPipeThreads;   // copies per thread
  extern __shared__ __align__(16) unsigned char fft_raw[];
  __shared__ float red[kPipeThreads / 32];
  float2 *stage = reinterpret_cast<float2 *>(fft_raw);  // [S][n][P]
  const int p = threadIdx.x & 31, t = threadIdx.x >> 5;
  const long long m = (long long)N * N;
  const int tpr = (N + P - 1) / P, total = N * tpr;
  // z0 and z1 share their layout (pitch even, 16-byte aligned rows); a bit per chunk whose
  // slice is read from z1
  unsigned from1 = 0;
  if (final_buf)
#pragma unroll
    for (int e = 0; e < kCh; e++) from1 |= (final_buf[(threadIdx.x + kPipeThreads * e) / (P / W)] ? 1u : 0u) << e;
  const float2 *b0 = reinterpret_cast<const float2 *>(z0.p), *b1 = reinterpret_cast<const float2 *>(z1.p);
  auto issue = [&](int tile, int st) {
    if (tile < total) {
      const int i = tile / tpr, c0 = (tile - i * tpr) * P;
      const uint32_t base = smem_u32(stage + (size_t)st * n * P);
#pragma unroll
      for (int e = 0; e < kCh; e++) {
        const int q = threadIdx.x + kPipeThreads * e, j = q / (P / W), pt = W * (q % (P / W));
        const bool ok = c0 + pt < N;  // a pair's second point may be the padding column
        // beyond the grid: zero fill from the row's last W-aligned point (no shared hot spot)
        const float2 *src = ((from1 >> e) & 1u ? b1 : b0) + (long long)j * z0.plane + (long long)i * z0.pitch +
                            min(c0 + pt, (N - 1) & ~(W - 1));
        cpa(base + (uint32_t)((j * P + pt) * sizeof(float2)), src, 8 * W, ok);
      }
    }
    cpa_commit();
  };
  float imax = 0.f;
  int q = 0;
  for (int s0 = 0; s0 < S - 1; s0++) issue(blockIdx.x + s0 * gridDim.x, s0);
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x, q++) {
    issue(tile + (S - 1) * gridDim.x, (q + S - 1) % S);
    const int i = tile / tpr, c = (tile - i * tpr) * P + p;
    const long long x = (long long)i * N + c;
    // the u values this thread accumulates into, requested before the stage wait and the
    // first pass so that their latency overlaps them
    double uo[N1];
    if (accumulate && c < N) {
#pragma unroll
      for (int r = 0; r < N1 / N2; r++)
#pragma unroll
        for (int k2 = 0; k2 < N2; k2++) uo[N2 * r + k2] = u[(long long)(t + N2 * r + N1 * k2) * m + x];
    }
    cpa_wait<S - 1>();
    __syncthreads();
    float2 *col = stage + (size_t)(q % S) * n * P;
    float2 v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; j1++) v[j1] = col[(N2 * j1 + t) * P + p];
    dft_small<float2, N1>(v, tw, N2);
#pragma unroll
    for (int k1 = 0; k1 < N1; k1++)
      col[(N2 * k1 + t) * P + p] = (k1 == 0 || t == 0) ? v[k1] : cmul(tw[(t * k1) % n], v[k1]);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < N1 / N2; r++) {
      const int k1 = t + N2 * r;
      float2 w[N2];
#pragma unroll
      for (int j2 = 0; j2 < N2; j2++) w[j2] = col[(N2 * k1 + j2) * P + p];
      dft_small<float2, N2>(w, tw, N1);
      if (c < N) {
#pragma unroll
        for (int k2 = 0; k2 < N2; k2++) {
          const int k = k1 + N1 * k2;
          const float wd = wk[k] * dscale;
          const float re = w[k2].x * wd;
          u[(long long)k * m + x] = accumulate ? uo[N2 * r + k2] + to_f64(re) : to_f64(re);
          if (imag_check) imax = fmaxf(imax, fabsf(w[k2].y * wd));
        }
      }
    }
    __syncthreads();  // the stage is refilled next
  }
  cpa_wait<0>();
  if (imag_check) {
    for (int o = 16; o > 0; o >>= 1) imax = fmaxf(imax, __shfl_down_sync(0xffffffffu, imax, o));
    if (p == 0) red[t] = imax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float mx = 0.f;
      for (int w = 0; w < kPipeThreads / 32; w++) mx = fmaxf(mx, red[w]);
      atomicMax(imag_bits, (unsigned long long)__double_as_longlong((double)mx));
    }
  }
}

template <int N1, typename InT> constexpr size_t fwd_pipe_smem() {
  return (size_t)(sizeof(InT) == 8 ? 2 : kPipeS) * N1 * kPipeTP * kPipeP * sizeof(InT) +
         (size_t)N1 * kPipeTP * kPipeP * sizeof(float2);
}
template <int N1> constexpr size_t inv_pipe_smem() { return (size_t)kPipeS * N1 * kPipeTP * kPipeP * sizeof(float2); }

// CTAs of a pipelined transform: as many as fit on the SMs at once (persistent), at most
// one per tile
template <typename K> int pipe_grid(K kernel, size_t smem, int N, int num_sms) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kPipeThreads, smem);
  const long long tiles = (long long)N * ((N + kPipeP - 1) / kPipeP);
  const long long g = (long long)(per < 1 ? 1 : per) * num_sms;
  return (int)(g < tiles ? g : tiles);
}

template <typename T, int n> size_t fft_smem() {
  return (size_t)n * fft_points<T, n>() * sizeof(typename Cx<T>::type);
}

int fft_grid(int N, int points, int num_sms) {
  const long long m = (long long)N * N;
  const long long ctas = (m + points - 1) / points;
  const long long cap = 8LL * num_sms;
  return (int)(ctas < cap ? ctas : cap);
}

template <typename T, int N1, int N2>
cudaError_t prepare_one() {
  const int bytes = (int)fft_smem<T, N1 * N2>();
  cudaError_t e = cudaFuncSetAttribute(k_fft_forward<T, N1, N2, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fft_forward<T, N1, N2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fft_inverse<T, N1, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

// the factorisations n = N1 N2 used for n = 2..128
#define PD_FFT_SIZES(X) X(2, 1) X(2, 2) X(4, 2) X(4, 4) X(8, 4) X(8, 8) X(16, 8)

}  // namespace

bool fft_transforms_supported(int n) { return n >= 2 && n <= 128 && (n & (n - 1)) == 0; }

template <int N1> cudaError_t prepare_pipe() {
  cudaError_t e = cudaFuncSetAttribute(k_fft_forward_pipe<N1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fwd_pipe_smem<N1, float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fft_forward_pipe<N1, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fwd_pipe_smem<N1, double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fft_inverse_pipe<N1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)inv_pipe_smem<N1>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fft_inverse_pipe<N1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)inv_pipe_smem<N1>());
}

template <typename T>
cudaError_t prepare_fft_transforms() {
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    e = prepare_pipe<8>();
    if (e == cudaSuccess) e = prepare_pipe<16>();
  }
#define PD_FFT_PREP(A, B)                      \
  if (e == cudaSuccess) e = prepare_one<T, A, B>();
  PD_FFT_SIZES(PD_FFT_PREP)
#undef PD_FFT_PREP
  return e;
}

// the pipelined FP32 kernels serve n = 64 and 128
template <int N1>
void launch_forward_pipe(cudaStream_t s, int num_sms, int N, View g, const void *f, bool f32,
                         const double *u0, const double *u0coef, const float *wk, const float2 *tw) {
  const long long tiles = (long long)N * ((N + kPipeP - 1) / kPipeP);
  if (f32) {
    constexpr size_t smem = fwd_pipe_smem<N1, float>();
    const int grid1 = pipe_grid(k_fft_forward_pipe<N1, float>, smem, 1 << 30, num_sms);
    k_fft_forward_pipe<N1, float><<<(int)std::min<long long>(grid1, tiles), kPipeThreads, smem, s>>>(
        N, g, static_cast<const float *>(f), u0, u0coef, wk, tw);
  } else {
    constexpr size_t smem = fwd_pipe_smem<N1, double>();
    const int grid1 = pipe_grid(k_fft_forward_pipe<N1, double>, smem, 1 << 30, num_sms);
    k_fft_forward_pipe<N1, double><<<(int)std::min<long long>(grid1, tiles), kPipeThreads, smem, s>>>(
        N, g, static_cast<const double *>(f), u0, u0coef, wk, tw);
  }
}

template <int N1>
void launch_inverse_pipe(cudaStream_t s, int num_sms, int N, double *u, View z0, View z1,
                         const int *final_buf, const float *wk, const float2 *tw, float dscale,
                         bool accumulate, bool imag_check, unsigned long long *imag_bits) {
  constexpr size_t smem = inv_pipe_smem<N1>();
  const long long tiles = (long long)N * ((N + kPipeP - 1) / kPipeP);
  // z1 is read only for the slices final_buf marks; both share the layout of z0
  const bool pairs = z0.pitch % 2 == 0 && z0.plane % 2 == 0 &&
                     reinterpret_cast<uintptr_t>(z0.p) % 16 == 0 && reinterpret_cast<uintptr_t>(z1.p) % 16 == 0;
  const int grid1 = pipe_grid(k_fft_inverse_pipe<N1, true>, smem, 1 << 30, num_sms);
  const int grid = (int)std::min<long long>(grid1, tiles);
  if (pairs)
    k_fft_inverse_pipe<N1, true><<<grid, kPipeThreads, smem, s>>>(
        N, u, z0, z1, final_buf, wk, tw, dscale, accumulate ? 1 : 0, imag_check ? 1 : 0, imag_bits);
  else
    k_fft_inverse_pipe<N1, false><<<grid, kPipeThreads, smem, s>>>(
        N, u, z0, z1, final_buf, wk, tw, dscale, accumulate ? 1 : 0, imag_check ? 1 : 0, imag_bits);
}

template <typename T>
void launch_fft_forward(cudaStream_t s, int num_sms, int N, int n, View g, const void *f, bool f32,
                        const double *u0, const double *u0coef, const T *wk,
                        const typename Cx<T>::type *tw) {
  if constexpr (sizeof(T) == 4) {
    if (n == 128) return launch_forward_pipe<16>(s, num_sms, N, g, f, f32, u0, u0coef, wk, tw);
    if (n == 64) return launch_forward_pipe<8>(s, num_sms, N, g, f, f32, u0, u0coef, wk, tw);
  }
#define PD_FFT_FWD(A, B)                                                                          \
  if (n == A * B) {                                                                               \
    constexpr int P = fft_points<T, A * B>(), TH = P * fft_tp<A, B, false>();                    \
    const int grid = fft_grid(N, P, num_sms);                                                     \
    const size_t smem = fft_smem<T, A * B>();                                                     \
    if (f32)                                                                                      \
      k_fft_forward<T, A, B, float><<<grid, TH, smem, s>>>(N, g, static_cast<const float *>(f),    \
                                                           u0, u0coef, wk, tw);                   \
    else                                                                                          \
      k_fft_forward<T, A, B, double><<<grid, TH, smem, s>>>(N, g, static_cast<const double *>(f),  \
                                                            u0, u0coef, wk, tw);                  \
    return;                                                                                       \
  }
  PD_FFT_SIZES(PD_FFT_FWD)
#undef PD_FFT_FWD
}

template <typename T>
void launch_fft_inverse(cudaStream_t s, int num_sms, int N, int n, double *u, View z0, View z1,
                        const int *final_buf, const T *wk, const typename Cx<T>::type *tw,
                        T dscale, bool accumulate, bool imag_check, unsigned long long *imag_bits) {
  if constexpr (sizeof(T) == 4) {
    if (n == 128)
      return launch_inverse_pipe<16>(s, num_sms, N, u, z0, z1, final_buf, wk, tw, dscale, accumulate,
                                     imag_check, imag_bits);
    if (n == 64)
      return launch_inverse_pipe<8>(s, num_sms, N, u, z0, z1, final_buf, wk, tw, dscale, accumulate,
                                    imag_check, imag_bits);
  }
#define PD_FFT_INV(A, B)                                                                       \
  if (n == A * B) {                                                                            \
    constexpr int P = fft_points<T, A * B>(), TH = P * fft_tp<A, B, true>();                  \
    const int grid = fft_grid(N, P, num_sms);                                                  \
    const size_t smem = fft_smem<T, A * B>();                                                  \
    k_fft_inverse<T, A, B><<<grid, TH, smem, s>>>(N, u, z0, z1, final_buf, wk, tw, dscale,     \
                                                 accumulate ? 1 : 0, imag_check ? 1 : 0,       \
                                                 imag_bits);                                   \
    return;                                                                                    \
  }
  PD_FFT_SIZES(PD_FFT_INV)
#undef PD_FFT_INV
}

#define PD_FFT_INST(T)                                                                            \
  template cudaError_t prepare_fft_transforms<T>();                                               \
  template void launch_fft_forward<T>(cudaStream_t, int, int, int, View, const void *, bool,     \
                                      const double *, const double *, const T *,                  \
                                      const typename Cx<T>::type *);                              \
  template void launch_fft_inverse<T>(cudaStream_t, int, int, int, double *, View, View,         \
                                      const int *, const T *, const typename Cx<T>::type *, T,    \
                                      bool, bool, unsigned long long *);
PD_FFT_INST(double)
PD_FFT_INST(float)

}  // namespace pd
