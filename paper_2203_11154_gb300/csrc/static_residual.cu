// pd_allatonce_residual_static: the residual check of the all-at-once system for the
// alpha-circulant backward-Euler step, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need this check: a host
// framework that owns all device memory through its own pool or arena and forbids
// other allocations, or a time-critical loop that cannot afford cudaMalloc's
// device-wide synchronisation.  This entry point takes every input and output from the
// caller and keeps its only scratch (per-CTA partial sums) in a fixed array in device
// global memory, declared below; it never allocates and needs no context.
#include <mutex>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kStaticMaxSteps = 128;    // largest n accepted
constexpr int kStaticBlocksPerStep = 64;
constexpr int kStaticThreads = 256;

// Partial sums of one call: [2][kStaticMaxSteps][kStaticBlocksPerStep] doubles (128 KiB).
// Every GPU that loads the library holds this array until the process exits.  Each call
// overwrites the partials it later reads, so nothing needs clearing; calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on it.
static __device__ __align__(256) double g_static_partials[2 * kStaticMaxSteps * kStaticBlocksPerStep];

// r_k = fhat_k - (u_k - u_{k-1}) / tau - A u_k, u_0 := alpha u_n, fhat_1 = f_1 + u0 / tau:
// CTA (b, k) sums r^2 and fhat^2 over its stride of row k into the scratch array.
__global__ void __launch_bounds__(kStaticThreads)
k_static_residual(int N, int n, double tau, double alpha, const double *__restrict__ u,
                  const double *__restrict__ f, const double *__restrict__ u0,
                  double *__restrict__ r, double *__restrict__ scratch) {
  __shared__ double red[2][kStaticThreads / 32];
  const int k = blockIdx.y;
  const long long m = (long long)N * N;
  const double h = 1.0 / (N + 1), ih2 = 1.0 / (h * h), itau = 1.0 / tau;
  const double *uk = u + (long long)k * m;
  const double *up = (k == 0) ? u + (long long)(n - 1) * m : u + (long long)(k - 1) * m;
  const double cprev = (k == 0) ? alpha : 1.0;
  double ar = 0.0, af = 0.0;
  for (long long x = (long long)blockIdx.x * kStaticThreads + threadIdx.x; x < m;
       x += (long long)gridDim.x * kStaticThreads) {
    const int i = (int)(x / N), c = (int)(x - (long long)i * N);
    double fh = f[(long long)k * m + x];
    if (k == 0 && u0) fh += u0[x] * itau;
    double nb = 0.0;
    if (i > 0) nb += uk[x - N];
    if (i < N - 1) nb += uk[x + N];
    if (c > 0) nb += uk[x - 1];
    if (c < N - 1) nb += uk[x + 1];
    const double rv = fh - (uk[x] - cprev * up[x]) * itau - ih2 * (4.0 * uk[x] - nb);
    if (r) r[(long long)k * m + x] = rv;
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
    for (int w = 0; w < kStaticThreads / 32; w++) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    const int slot = k * kStaticBlocksPerStep + blockIdx.x;
    scratch[slot] = s0;
    scratch[kStaticMaxSteps * kStaticBlocksPerStep + slot] = s1;
  }
}

// norms[0] = ||r||_2, norms[1] = ||fhat||_2 from the partials, in a fixed order.
__global__ void k_static_norms(int n, const double *__restrict__ scratch, double *__restrict__ norms) {
  __shared__ double red[2][32];
  const int lane = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int s = lane; s < n * kStaticBlocksPerStep; s += 32) {
    a += scratch[s];
    b += scratch[kStaticMaxSteps * kStaticBlocksPerStep + s];
  }
  red[0][lane] = a;
  red[1][lane] = b;
  __syncwarp();
  if (lane == 0) {
    double sa = 0.0, sb = 0.0;
    for (int q = 0; q < 32; q++) {
      sa += red[0][q];
      sb += red[1][q];
    }
    norms[0] = sqrt(sa);
    norms[1] = sqrt(sb);
  }
}

// Device address of the scratch array, looked up once per device (with that device
// current) and cached.
constexpr int kMaxDevices = 64;
std::mutex g_symbol_mutex;
void *g_symbol_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_symbol_mutex);
  if (!g_symbol_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess) return e;
    g_symbol_ptr[dev] = p;
  }
  *out = static_cast<double *>(g_symbol_ptr[dev]);
  return cudaSuccess;
}

}  // namespace
}  // namespace pd

extern "C" pd_status pd_allatonce_residual_static(int N, int n, double tau, double alpha,
                                                  const double *d_u, const double *d_f,
                                                  const double *d_u0, double *d_r,
                                                  double *d_norms, void *stream) {
  using namespace pd;
  if (N < 1 || n < 1 || !(tau > 0) || !(alpha > 0) || alpha > 1 || !d_u || !d_f || !d_norms)
    return PD_ERR_ARG;
  if (n > kStaticMaxSteps) return PD_ERR_ARG;  // the scratch array holds 128 time steps
  double *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return PD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_static_residual<<<dim3(kStaticBlocksPerStep, n), kStaticThreads, 0, s>>>(N, n, tau, alpha, d_u,
                                                                             d_f, d_u0, d_r, scratch);
  k_static_norms<<<1, 32, 0, s>>>(n, scratch, d_norms);
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ERR_CUDA;
}
