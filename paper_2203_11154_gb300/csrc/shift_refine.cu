// FP64 refinement of the shifted systems of eq. (2) around the FP32 multigrid: the FP64
// residual of each system, handed to the FP32 levels as the next right-hand side, and the
// FP64 update of the solution with the FP32 correction.
//
//   r_j = b_j - (lam_j I + kappa A) z_j,  A the five-point Laplacian (1/h^2)[4, -1 x 4]
//
// written per point as r = b - c1 z + off * (sum of the 4 neighbours of z), c1 = lam_j +
// 4 kappa/h^2 and off = kappa/h^2, in FP64 complex; the FP32 copy handed to the multigrid
// is scaled by h^2/kappa, the scaling of the level-0 right-hand side.
#include "cplx.cuh"
#include "fpbits.cuh"
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kSrThreads = 256;

// grid (gx, n): CTA x of shift j strides over the grid rows of shift j.  The FP32 output
// is sc_j r (sc_j a power of two that keeps the shift's FP32 right-hand side near unit
// size) times oscale; part[j][x] gets the CTA's sum of |sc_j r|^2 (and of |b|^2, in FP64,
// in part[n + j][x] when want_b); frozen shifts (already converged) get a zero right-hand
// side and no sums.
__global__ void __launch_bounds__(kSrThreads)
k_shift_residual(int N, const double2 *__restrict__ z, const double2 *__restrict__ b,
                 const double2 *__restrict__ c1, double off, float oscale, const float *__restrict__ sc,
                 View out, const int *__restrict__ frozen, int want_b, double *__restrict__ part) {
  __shared__ double red[2][kSrThreads / 32];
  const int j = blockIdx.y;
  const long long m = (long long)N * N;
  const bool fz = frozen && frozen[j];
  const double2 cj = c1[j];
  const int sce = (int)((__float_as_uint(sc[j]) >> 23) & 0xFFu) - 127;  // sc_j = 2^sce
  float2 *o = reinterpret_cast<float2 *>(out.p) + (long long)j * out.plane;
  double ar = 0.0, ab = 0.0;
  for (int i = blockIdx.x; i < N; i += gridDim.x) {
    const double2 *br = b + j * m + (long long)i * N;
    const double2 *zr = z ? z + j * m + (long long)i * N : nullptr;
    float rowr = 0.f;
    double rowb = 0.0;
    for (int c = threadIdx.x; c < N; c += kSrThreads) {
      if (fz) {
        o[(long long)i * out.pitch + c] = make_float2(0.f, 0.f);
        continue;
      }
      const double2 bv = br[c];
      double2 r = bv;
      if (zr) {
        double2 nb = make_double2(0.0, 0.0);
        if (c > 0) nb = cadd(nb, zr[c - 1]);
        if (c < N - 1) nb = cadd(nb, zr[c + 1]);
        if (i > 0) nb = cadd(nb, zr[c - N]);
        if (i < N - 1) nb = cadd(nb, zr[c + N]);
        const double2 zv = zr[c];
        // r = b - c1 z + off nb
        r.x = fma(off, nb.x, fma(-cj.x, zv.x, fma(cj.y, zv.y, bv.x)));
        r.y = fma(off, nb.y, fma(-cj.x, zv.y, fma(-cj.y, zv.x, bv.y)));
      }
      const float2 rf = make_float2(f64_to_f32(r.x, sce), f64_to_f32(r.y, sce));
      rowr = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, rowr));
      if (want_b) rowb = fma(bv.x, bv.x, fma(bv.y, bv.y, rowb));
      o[(long long)i * out.pitch + c] = make_float2(rf.x * oscale, rf.y * oscale);
    }
    ar += (double)rowr;
    ab += rowb;
  }
  for (int s = 16; s > 0; s >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, s);
    ab += __shfl_down_sync(0xffffffffu, ab, s);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ar;
    red[1][threadIdx.x >> 5] = ab;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kSrThreads / 32; w++) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[(long long)j * gridDim.x + blockIdx.x] = s0;
    if (want_b) part[(long long)(gridDim.y + j) * gridDim.x + blockIdx.x] = s1;
  }
}

// z_j (+)= d_j / sc_j for the shifts that are not frozen; d_j is the FP32 answer of the
// multigrid in z0 or z1 (final_buf[j]) for the right-hand side scaled by sc_j
__global__ void k_shift_update(int N, double2 *__restrict__ z, View z0, View z1,
                               const int *__restrict__ final_buf, const int *__restrict__ frozen,
                               const float *__restrict__ sc, int accumulate) {
  const int j = blockIdx.z;
  if (frozen && frozen[j]) return;
  const int i = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 32 + threadIdx.x;
  if (i >= N || c >= N) return;
  const View &src = final_buf[j] ? z1 : z0;
  const float isc = 1.0f / sc[j];  // a power of two: exact
  float2 d =
      reinterpret_cast<const float2 *>(src.p)[(long long)j * src.plane + (long long)i * src.pitch + c];
  d.x *= isc;
  d.y *= isc;
  double2 &dst = z[(long long)j * N * N + (long long)i * N + c];
  if (accumulate) {
    dst.x += f32_to_f64(d.x);
    dst.y += f32_to_f64(d.y);
  } else {
    dst = make_double2(f32_to_f64(d.x), f32_to_f64(d.y));
  }
}

__global__ void k_round_to_float(long long count, const double *__restrict__ x, float *__restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// dst = src, 16 bytes a thread and step, with streaming (evict-first) loads and stores:
// the device-to-host copy of a result into mapped pinned memory, run beside a solve, then
// displaces less of the solve's L2 working set than a copy-engine transfer does
__global__ void k_stream_copy(const float4 *__restrict__ src, float4 *__restrict__ dst, long long n16) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16;
       i += (long long)gridDim.x * blockDim.x)
    __stcs(dst + i, __ldcs(src + i));
}

}  // namespace

void launch_stream_copy(cudaStream_t s, int blocks, const void *src, void *dst, long long n16) {
  k_stream_copy<<<blocks, 512, 0, s>>>(static_cast<const float4 *>(src), static_cast<float4 *>(dst), n16);
}

void launch_round_to_float(cudaStream_t s, long long count, const double *x, float *y) {
  const long long blocks = (count + 255) / 256;
  k_round_to_float<<<(int)(blocks < 1 ? 1 : (blocks > 65535 ? 65535 : blocks)), 256, 0, s>>>(count, x, y);
}

void launch_shift_residual(cudaStream_t s, int gx, int N, int n, const double2 *z, const double2 *b,
                           const double2 *c1, double off, float oscale, const float *sc, View out,
                           const int *frozen, bool want_b, double *part) {
  dim3 grid(gx, n);
  k_shift_residual<<<grid, kSrThreads, 0, s>>>(N, z, b, c1, off, oscale, sc, out, frozen,
                                               want_b ? 1 : 0, part);
}

void launch_shift_update(cudaStream_t s, int N, int n, double2 *z, View z0, View z1,
                         const int *final_buf, const int *frozen, const float *sc, bool accumulate) {
  dim3 grid((N + 31) / 32, (N + 7) / 8, n);
  k_shift_update<<<grid, dim3(32, 8), 0, s>>>(N, z, z0, z1, final_buf, frozen, sc, accumulate ? 1 : 0);
}

}  // namespace pd
