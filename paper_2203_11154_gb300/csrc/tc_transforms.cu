// Time-direction transforms of eq. (1) on the 5th-generation tensor cores (tcgen05),
// for n <= 128 shifts (the forms for 64 < n <= 128 are described where they are defined).  Both are real GEMMs D[128 x Nt] = A[128 x K] B[K x Nt] over tiles
// of Nt grid points of one grid row, in TF32 with the 3-product split
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,  x_hi = x rounded to TF32, x_lo = x - x_hi,
// accumulated in FP32 in tensor memory: about 2^-21 relative per product, the
// FP32-compensated product the refinement needs because V can be ill-conditioned.
//
//   forward:  K = 64 (k < n),  rows 2j / 2j+1 of A = Re / Im of h^2 V^{-1}[j][k],
//             B[k][p] = fhat_k at point p (FP64 or FP32 input, rounded to FP32 then split);
//             g_j(p) = (D[2j][p], D[2j+1][p]).
//   inverse:  K = 128 (2j + re/im), row k of A = (Re V[k][j], -Im V[k][j]) and row 64 + k =
//             (Im V[k][j], Re V[k][j]), B[2j+q][p] = component q of z_j(p);
//             u_k(p) (+)= D[k][p], max |D[64+k][p]| is the imaginary-part check.
//
// Operands live in shared memory in the K-major layout with 128-byte swizzling (8-row x
// 128-byte atoms, 16-byte chunk c of row r stored at chunk c ^ (r mod 8)); A is loaded
// once per CTA, B is built per tile by all threads.  One thread issues the MMAs and
// commits them to an mbarrier; the epilogue reads the accumulators with tcgen05.ld
// through a padded shared-memory stage so that the global stores are coalesced.
#include "cplx.cuh"
#include "pd_internal.h"
#include "tma.cuh"

#include <algorithm>

namespace pd {
namespace {

constexpr int kTcThreads = 256;
constexpr int kM = 128;

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1 << 16;                   // leading-dimension offset (unused: swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride between 8-row groups: 8 x 128 B
  d |= (uint64_t)1 << 46;                   // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; q++) v[q] = __uint_as_float(r[q]);
}

// TF32 split: hi = x rounded to 10 explicit mantissa bits, lo = x - hi (exact)
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  const uint32_t b = (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
  hi = __uint_as_float(b);
  lo = x - hi;
}

// byte offset of the 16-byte chunk holding K values [4q, 4q+4) of row `row` in a
// K-major, 128B-swizzled operand with `rows` rows
__device__ __forceinline__ uint32_t sw_off(int row, int q, int rows) {
  const int atom = q >> 3, ch = q & 7;
  return (uint32_t)(atom * rows * 128 + row * 128 + ((ch ^ (row & 7)) << 4));
}

// copies a row-major [128][K] float matrix from global memory into the swizzled layout
template <int K>
__device__ void load_a(const float *__restrict__ src, unsigned char *dst) {
  for (int it = threadIdx.x; it < kM * (K / 4); it += kTcThreads) {
    const int row = it / (K / 4), q = it % (K / 4);
    const float4 v = *reinterpret_cast<const float4 *>(src + (size_t)row * K + 4 * q);
    *reinterpret_cast<float4 *>(dst + sw_off(row, q, kM)) = v;
  }
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// issues the 3 x (K/8) MMAs of one tile and commits them to `bar` (one thread)
template <int K, int NT>
__device__ __forceinline__ void issue_tile(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                           uint32_t b_lo, uint64_t *bar) {
  constexpr uint32_t idesc = idesc_tf32(kM, NT);
  uint32_t acc = 0;
#pragma unroll
  for (int ks = 0; ks < K / 8; ks++) {
    const uint32_t ao = (uint32_t)((ks >> 2) * kM * 128 + (ks & 3) * 32);
    const uint32_t bo = (uint32_t)((ks >> 2) * NT * 128 + (ks & 3) * 32);
    mma_tf32(tmem, desc_sw128(a_hi + ao), desc_sw128(b_hi + bo), idesc, acc);
    acc = 1;
    mma_tf32(tmem, desc_sw128(a_hi + ao), desc_sw128(b_lo + bo), idesc, 1);
    mma_tf32(tmem, desc_sw128(a_lo + ao), desc_sw128(b_hi + bo), idesc, 1);
  }
  mma_commit(bar);
}

constexpr int kFwdK = 64, kFwdNt = 128, kInvK = 128, kInvNt = 64;
constexpr int kFwdA = kM * kFwdK * 4, kFwdB = kFwdNt * kFwdK * 4;  // bytes per split
constexpr int kInvA = kM * kInvK * 4, kInvB = kInvNt * kInvK * 4;
constexpr int kFwdS = 64 * 66 * 4;   // epilogue stage: 64 j rows x 32 complex (stride 66 floats)
constexpr int kInvS = kM * (kInvNt + 1) * 4;  // epilogue stage: 128 rows x 64 columns (stride 65)
constexpr int kFwdSmem = 2 * kFwdA + 2 * kFwdB + kFwdS + 1024;
constexpr int kInvSmem = 2 * kInvA + 2 * kInvB + kInvS + 1024;

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return p + ((1024 - (smem_u32(p) & 1023)) & 1023);
}

// g_j(p) = h^2 sum_k V^{-1}[j][k] fhat_k(p), fhat_k = in_scale (f_k + u0coef[k] u0), for the
// points p = (i, c0..c0+NT-1) of grid row i; written into the h^2-scaled level-0 RHS view
// (in_scale: a power of two that brings the refinement's FP64 residual near unit size).
// The rows of A are (Re, Im) of 64 shifts: with HALVES = 2 (n <= 128, K = 128) CTA x takes
// the shifts 64 (x mod 2) .. + 63, its A the matching half of the operand, and the tiles
// x / 2, x / 2 + gridDim.x / 2, ... (the two CTAs of a tile read its input once from DRAM).
template <typename InT, int K, int NT, int HALVES>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_forward(int N, int n, View g, const InT *__restrict__ f, const double *__restrict__ u0,
             const double *__restrict__ u0coef, const float *__restrict__ Ahi,
             const float *__restrict__ Alo, double in_scale, int *__restrict__ errflag) {
  constexpr int kA = kM * K * 4, kB = NT * K * 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = align1024(smem_raw);
  unsigned char *sAhi = sm, *sAlo = sm + kA, *sBhi = sm + 2 * kA, *sBlo = sBhi + kB;
  float *S = reinterpret_cast<float *>(sBlo + kB);
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = (int)blockIdx.x % HALVES, jbase = 64 * half;
  const int t0 = (int)blockIdx.x / HALVES, tstep = (int)gridDim.x / HALVES;
  if (warp == 0) tmem_alloc(&tmem_slot, NT);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  load_a<K>(Ahi + (size_t)half * kM * K, sAhi);
  load_a<K>(Alo + (size_t)half * kM * K, sAlo);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const long long m = (long long)N * N;
  const int tpr = (int)((g.pitch + NT - 1) / NT);  // tiles per grid row
  const int total = N * tpr;
  const int nj = min(64, n - jbase);  // shifts of this CTA
  uint32_t phase = 0;
  bool ok = true;
  // each thread owns kFwdItems (point, 4 consecutive k) items of a tile; the FP64 inputs of
  // the next tile are loaded into registers while the current tile is multiplied
  constexpr int kFwdItems = NT * (K / 4) / kTcThreads;
  // held in FP32 (the operand precision); FP64 arithmetic only for the initial-value
  // term of the rows where it is nonzero (GB300's FP64 rate is 1/58 of FP32)
  float pre[kFwdItems][4];
  auto fetch = [&](int t) {
    const int i = t / tpr, c0 = (t % tpr) * NT;
#pragma unroll
    for (int q = 0; q < kFwdItems; q++) {
      const int it = tid + q * kTcThreads;
      const int p = it % NT, kq = it / NT;
      const int c = c0 + p;
      const long long x = (long long)i * N + c;
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int k = 4 * kq + e;
        float v = 0.f;
        if (k < n && c < N) {
          const double ck = u0 ? u0coef[k] : 0.0;
          if (ck != 0.0) v = (float)(((double)f[k * m + x] + ck * u0[x]) * in_scale);
          else if (in_scale != 1.0) v = (float)((double)f[k * m + x] * in_scale);
          else v = (float)f[k * m + x];
        }
        pre[q][e] = v;
      }
    }
  };
  int t = t0;
  if (t < total) fetch(t);
  for (; t < total; t += tstep) {
    const int i = t / tpr, c0 = (t % tpr) * NT;
    // B[p][k] = fhat_k(i, c0 + p), split into TF32 hi/lo, 16-byte swizzled chunks
#pragma unroll
    for (int q = 0; q < kFwdItems; q++) {
      const int it = tid + q * kTcThreads;
      const int p = it % NT, kq = it / NT;
      float4 hi, lo;
      split_tf32(pre[q][0], hi.x, lo.x);
      split_tf32(pre[q][1], hi.y, lo.y);
      split_tf32(pre[q][2], hi.z, lo.z);
      split_tf32(pre[q][3], hi.w, lo.w);
      *reinterpret_cast<float4 *>(sBhi + sw_off(p, kq, NT)) = hi;
      *reinterpret_cast<float4 *>(sBlo + sw_off(p, kq, NT)) = lo;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_tile<K, NT>(tmem, smem_u32(sAhi), smem_u32(sAlo), smem_u32(sBhi), smem_u32(sBlo),
                                &bar);
    }
    if (t + tstep < total) fetch(t + tstep);
    ok = mbar_wait_bounded(&bar, phase);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(errflag, 4);
      break;
    }
    phase ^= 1;
    tc_fence_after();
    // epilogue, 32 columns at a time: lanes of warps 0-3 hold rows 2j+q of D
    for (int chunk = 0; chunk < NT / 32; chunk++) {
      if (warp < 4) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * chunk), v);
        const int row = 32 * warp + lane, j = row >> 1, q = row & 1;
        if (j < nj)
#pragma unroll
          for (int cc = 0; cc < 32; cc++) S[j * 66 + 2 * cc + q] = v[cc];
      }
      __syncthreads();
      for (int it = tid; it < nj * 32; it += kTcThreads) {
        const int j = it >> 5, cc = it & 31;
        const int c = c0 + 32 * chunk + cc;
        if (c < N) {
          const float2 val = *reinterpret_cast<const float2 *>(&S[j * 66 + 2 * cc]);
          reinterpret_cast<float2 *>(g.p)[(jbase + j) * g.plane + (long long)i * g.pitch + c] = val;
        }
      }
      __syncthreads();
    }
    tc_fence_before();
  }
  if (!ok && tid == 0) mbar_wait_bounded(&bar, phase);  // let an MMA in flight finish
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, NT);
}

// u_k(p) (+)= Re sum_j V[k][j] z_j(p) for p = (i, c0..c0+63); z_j is read from z1 where
// final_buf[j] is set, else from z0; imag_check: atomic max of |Im| (bits of a double).
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_inverse(int N, int n, double *__restrict__ u, View z0, View z1, const int *__restrict__ final_buf,
             const float *__restrict__ Ahi, const float *__restrict__ Alo, float dscale, int accumulate,
             int imag_check, unsigned long long *imag_bits, int *__restrict__ errflag) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = align1024(smem_raw);
  unsigned char *sAhi = sm, *sAlo = sm + kInvA, *sBhi = sm + 2 * kInvA, *sBlo = sBhi + kInvB;
  float *S = reinterpret_cast<float *>(sBlo + kInvB);
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float red[kTcThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_slot, kInvNt);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  load_a<kInvK>(Ahi, sAhi);
  load_a<kInvK>(Alo, sAlo);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const long long m = (long long)N * N;
  const int tpr = (int)((z0.pitch + kInvNt - 1) / kInvNt);
  const int total = N * tpr;
  uint32_t phase = 0;
  bool ok = true;
  float imax = 0.f;
  // each thread owns kInvItems (point, 2 shifts) items of a tile; the z values of the
  // next tile are loaded into registers while the current tile is multiplied
  constexpr int kInvItems = kInvNt * (kInvK / 4) / kTcThreads;
  float2 pre[kInvItems][2];
  auto fetch = [&](int t) {
    const int i = t / tpr, c0 = (t % tpr) * kInvNt;
#pragma unroll
    for (int q = 0; q < kInvItems; q++) {
      const int it = tid + q * kTcThreads;
      const int p = it % kInvNt, qq = it / kInvNt;
      const int c = c0 + p;
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int jj = 2 * qq + e;
        float2 v = make_float2(0.f, 0.f);
        if (c < N && jj < n) {
          const View &zv = (final_buf && final_buf[jj]) ? z1 : z0;
          v = reinterpret_cast<const float2 *>(zv.p)[jj * zv.plane + (long long)i * zv.pitch + c];
        }
        pre[q][e] = v;
      }
    }
  };
  // u values this thread accumulates into in the epilogue (n x 64 per tile)
  constexpr int kAccItems = 64 * kInvNt / kTcThreads;
  double uacc[kAccItems];
  int t = blockIdx.x;
  if (t < total) fetch(t);
  for (; t < total; t += gridDim.x) {
    const int i = t / tpr, c0 = (t % tpr) * kInvNt;
#pragma unroll
    for (int q = 0; q < kInvItems; q++) {
      const int it = tid + q * kTcThreads;
      const int p = it % kInvNt, qq = it / kInvNt;
      float4 hi, lo;
      split_tf32(pre[q][0].x, hi.x, lo.x);
      split_tf32(pre[q][0].y, hi.y, lo.y);
      split_tf32(pre[q][1].x, hi.z, lo.z);
      split_tf32(pre[q][1].y, hi.w, lo.w);
      *reinterpret_cast<float4 *>(sBhi + sw_off(p, qq, kInvNt)) = hi;
      *reinterpret_cast<float4 *>(sBlo + sw_off(p, qq, kInvNt)) = lo;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_tile<kInvK, kInvNt>(tmem, smem_u32(sAhi), smem_u32(sAlo), smem_u32(sBhi), smem_u32(sBlo),
                                &bar);
    }
    // accumulator inputs of this tile and z of the next one, while the MMAs run
#pragma unroll
    for (int q = 0; q < kAccItems; q++) {
      const int it = tid + q * kTcThreads;
      const int k = it / kInvNt, cc = it % kInvNt;
      const int c = c0 + cc;
      uacc[q] = (accumulate && k < n && c < N) ? u[(long long)k * m + (long long)i * N + c] : 0.0;
    }
    if (t + (int)gridDim.x < total) fetch(t + gridDim.x);
    ok = mbar_wait_bounded(&bar, phase);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(errflag, 4);
      break;
    }
    phase ^= 1;
    tc_fence_after();
    for (int chunk = 0; chunk < kInvNt / 32; chunk++) {
      if (warp < 4) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * chunk), v);
        const int row = 32 * warp + lane;
#pragma unroll
        for (int cc = 0; cc < 32; cc++) S[row * (kInvNt + 1) + 32 * chunk + cc] = v[cc];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kAccItems; q++) {
      const int it = tid + q * kTcThreads;
      const int k = it / kInvNt, cc = it % kInvNt;
      const int c = c0 + cc;
      if (k < n && c < N) {
        u[(long long)k * m + (long long)i * N + c] = uacc[q] + (double)(S[k * (kInvNt + 1) + cc] * dscale);
        if (imag_check) imax = fmaxf(imax, fabsf(S[(64 + k) * (kInvNt + 1) + cc] * dscale));
      }
    }
    __syncthreads();
    tc_fence_before();
  }
  if (!ok && tid == 0) mbar_wait_bounded(&bar, phase);
  if (imag_check) {
    for (int o = 16; o > 0; o >>= 1) imax = fmaxf(imax, __shfl_down_sync(0xffffffffu, imax, o));
    if (lane == 0) red[warp] = imax;
  }
  __syncthreads();
  if (imag_check && tid == 0) {
    float mx = 0.f;
    for (int w = 0; w < kTcThreads / 32; w++) mx = fmaxf(mx, red[w]);
    atomicMax(imag_bits, (unsigned long long)__double_as_longlong((double)mx));
  }
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kInvNt);
}

// ---- the inverse for 64 < n <= 128: K = 2n split over the two CTAs of a cluster ----
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// all threads of both CTAs of the cluster; release/acquire orders shared::cluster stores
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the shared::cluster address of this CTA's shared-memory address `saddr` in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

constexpr int kInv2K = 128, kInv2Nt = 32;
constexpr int kInv2A = kM * kInv2K * 4, kInv2B = kInv2Nt * kInv2K * 4;
constexpr int kInv2S = kM * (kInv2Nt + 1) * 4;
constexpr int kInv2Smem = 2 * kInv2A + 2 * kInv2B + kInv2S + 1024;

// u_k(p) (+)= dscale Re sum_j V[k][j] z_j(p) for k < 128 and the points p = (i, c0..c0+31):
// CTA r of a cluster of two multiplies the shifts j = 64 r .. 64 r + 63 (its half of K,
// A = its half of the operand), both accumulate D[128 x 32] in tensor memory; CTA 1 stores
// its D into CTA 0's stage through distributed shared memory, CTA 0 adds its own and writes
// u.  The imaginary part is not formed on this route.  Both CTAs of a cluster walk the same
// tiles and meet at every cluster barrier, also after a bounded wait ran out (then they only
// skip the work), so neither can wait for the other forever.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTcThreads, 1)
k_tc_inverse2(int N, int n, double *__restrict__ u, View z0, View z1, const int *__restrict__ final_buf,
              const float *__restrict__ Ahi, const float *__restrict__ Alo, float dscale, int accumulate,
              int *__restrict__ errflag) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = align1024(smem_raw);
  unsigned char *sAhi = sm, *sAlo = sm + kInv2A, *sBhi = sm + 2 * kInv2A, *sBlo = sBhi + kInv2B;
  float *S = reinterpret_cast<float *>(sBlo + kInv2B);
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const int jbase = 64 * (int)rank;
  if (warp == 0) tmem_alloc(&tmem_slot, kInv2Nt);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  load_a<kInv2K>(Ahi + (size_t)rank * kM * kInv2K, sAhi);
  load_a<kInv2K>(Alo + (size_t)rank * kM * kInv2K, sAlo);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t S_peer = peer_addr(smem_u32(S), 0);  // CTA 0's stage
  const long long m = (long long)N * N;
  const int tpr = (int)((z0.pitch + kInv2Nt - 1) / kInv2Nt);
  const int total = N * tpr;
  const int t0 = (int)blockIdx.x / 2, tstep = (int)gridDim.x / 2;
  uint32_t phase = 0;
  bool ok = true;
  // each thread owns kItems (point, 2 shifts) items of a tile; the z values of the next
  // tile are loaded into registers while the current tile is multiplied
  constexpr int kItems = kInv2Nt * (kInv2K / 4) / kTcThreads;
  float2 pre[kItems][2];
  auto fetch = [&](int t) {
    const int i = t / tpr, c0 = (t % tpr) * kInv2Nt;
#pragma unroll
    for (int q = 0; q < kItems; q++) {
      const int it = tid + q * kTcThreads;
      const int p = it % kInv2Nt, qq = it / kInv2Nt;
      const int c = c0 + p;
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int jj = jbase + 2 * qq + e;
        float2 v = make_float2(0.f, 0.f);
        if (c < N && jj < n) {
          const View &zv = (final_buf && final_buf[jj]) ? z1 : z0;
          v = reinterpret_cast<const float2 *>(zv.p)[jj * zv.plane + (long long)i * zv.pitch + c];
        }
        pre[q][e] = v;
      }
    }
  };
  constexpr int kAcc = kM * kInv2Nt / kTcThreads;  // u values of a tile per thread (CTA 0)
  double uacc[kAcc];
  int t = t0;
  if (t < total) fetch(t);
  for (; t < total; t += tstep) {
    const int i = t / tpr, c0 = (t % tpr) * kInv2Nt;
    if (ok) {
#pragma unroll
      for (int q = 0; q < kItems; q++) {
        const int it = tid + q * kTcThreads;
        const int p = it % kInv2Nt, qq = it / kInv2Nt;
        float4 hi, lo;
        split_tf32(pre[q][0].x, hi.x, lo.x);
        split_tf32(pre[q][0].y, hi.y, lo.y);
        split_tf32(pre[q][1].x, hi.z, lo.z);
        split_tf32(pre[q][1].y, hi.w, lo.w);
        *reinterpret_cast<float4 *>(sBhi + sw_off(p, qq, kInv2Nt)) = hi;
        *reinterpret_cast<float4 *>(sBlo + sw_off(p, qq, kInv2Nt)) = lo;
      }
      fence_proxy_async_smem();
      tc_fence_before();
    }
    __syncthreads();
    if (ok && tid == 0) {
      tc_fence_after();
      issue_tile<kInv2K, kInv2Nt>(tmem, smem_u32(sAhi), smem_u32(sAlo), smem_u32(sBhi), smem_u32(sBlo), &bar);
    }
    if (rank == 0) {
#pragma unroll
      for (int q = 0; q < kAcc; q++) {
        const int it = tid + q * kTcThreads;
        const int k = it / kInv2Nt, c = c0 + it % kInv2Nt;
        uacc[q] = (accumulate && k < n && c < N) ? u[(long long)k * m + (long long)i * N + c] : 0.0;
      }
    }
    if (t + tstep < total) fetch(t + tstep);
    if (ok) {
      const bool w = mbar_wait_bounded(&bar, phase);
      ok = __syncthreads_and(w);
      if (!ok && tid == 0) atomicOr(errflag, 4);
      if (w) phase ^= 1;
    } else {
      __syncthreads();
    }
    tc_fence_after();
    cluster_sync();  // CTA 0's stage is free
    if (rank == 1 && ok && warp < 4) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
      const int row = 32 * warp + lane;
#pragma unroll
      for (int cc = 0; cc < 32; cc++) st_cluster(S_peer + (uint32_t)((row * (kInv2Nt + 1) + cc) * 4), v[cc]);
    }
    cluster_sync();  // CTA 1's half of D is in CTA 0's stage
    if (rank == 0) {
      if (ok && warp < 4) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
        const int row = 32 * warp + lane;
#pragma unroll
        for (int cc = 0; cc < 32; cc++) S[row * (kInv2Nt + 1) + cc] += v[cc];
      }
      __syncthreads();
      if (ok) {
#pragma unroll
        for (int q = 0; q < kAcc; q++) {
          const int it = tid + q * kTcThreads;
          const int k = it / kInv2Nt, cc = it % kInv2Nt, c = c0 + cc;
          if (k < n && c < N)
            u[(long long)k * m + (long long)i * N + c] = uacc[q] + (double)(S[k * (kInv2Nt + 1) + cc] * dscale);
        }
      }
    }
    __syncthreads();
    tc_fence_before();
  }
  if (!ok && tid == 0) mbar_wait_bounded(&bar, phase);  // let an MMA in flight finish
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kInv2Nt);
  cluster_sync();  // CTA 0's shared memory stays until CTA 1 is done with it
}

}  // namespace

bool tc_transforms_supported(int N, int n) { return n <= 128 && N >= 127; }

// the forward for 64 < n <= 128: K = 128, tiles of 64 points, two CTAs (halves of the rows)
constexpr int kFwd2K = 128, kFwd2Nt = 64;
constexpr int kFwd2Smem = 2 * kM * kFwd2K * 4 + 2 * kFwd2Nt * kFwd2K * 4 + kFwdS + 1024;
static_assert(kFwd2Smem <= 227 * 1024 - 256, "forward operands exceed shared memory");
static_assert(kInv2Smem <= 227 * 1024 - 256, "inverse operands exceed shared memory");

cudaError_t prepare_tc_transforms() {
  cudaError_t e;
#define PD_TC_ATTR(K_, S_)                                                         \
  e = cudaFuncSetAttribute(K_, cudaFuncAttributeMaxDynamicSharedMemorySize, S_); \
  if (e != cudaSuccess) return e;
  PD_TC_ATTR((k_tc_forward<double, kFwdK, kFwdNt, 1>), kFwdSmem)
  PD_TC_ATTR((k_tc_forward<float, kFwdK, kFwdNt, 1>), kFwdSmem)
  PD_TC_ATTR((k_tc_forward<double, kFwd2K, kFwd2Nt, 2>), kFwd2Smem)
  PD_TC_ATTR((k_tc_forward<float, kFwd2K, kFwd2Nt, 2>), kFwd2Smem)
  PD_TC_ATTR(k_tc_inverse, kInvSmem)
  PD_TC_ATTR(k_tc_inverse2, kInv2Smem)
#undef PD_TC_ATTR
  return cudaSuccess;
}

// A operands (host): TF32 splits of the scaled forward matrix [128][64] and of the
// inverse matrix [128][128] in the row layouts described at the top of this file.
static void split_host(double x, float &hi, float &lo) {
  const float xf = (float)x;
  uint32_t b;
  memcpy(&b, &xf, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  memcpy(&hi, &b, 4);
  lo = (float)(x - (double)hi);
}

// CTAs of a launch: one per SM (one CTA fits an SM); for n > 64 an even count, the inverse's
// pairs as many as the device can hold at once as two-CTA clusters (a GPC with an odd count
// of free SMs leaves one idle), so that no cluster waits for a second wave
cudaError_t tc_launch_grid(int num_sms, int n, bool inverse, int *grid) {
  if (n <= 64) {
    *grid = num_sms;
    return cudaSuccess;
  }
  if (!inverse) {
    *grid = std::max(2, num_sms & ~1);
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(kTcThreads, 1, 1);
  cfg.dynamicSmemBytes = kInv2Smem;
  int clusters = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, k_tc_inverse2, &cfg);
  if (e != cudaSuccess) return e;
  *grid = 2 * std::max(1, std::min(clusters, num_sms / 2));
  return cudaSuccess;
}

size_t tc_operand_floats(int n, bool inverse) {
  if (n <= 64) return inverse ? (size_t)kM * kInvK : (size_t)kM * kFwdK;
  return 2 * (size_t)kM * (inverse ? kInv2K : kFwd2K);
}

void tc_build_operands(int n, const double *Vinv, const double *V, double scale, float *fwd_hi,
                       float *fwd_lo, float *inv_hi, float *inv_lo) {
  if (n > 64) {
    // two halves: forward rows 2 jl + q of shift j = 64 h + jl, K = time step k; inverse
    // rows k (real part only), K = 2 jl + q of shift j = 64 h + jl
    for (int h = 0; h < 2; h++)
      for (int r = 0; r < kM; r++)
        for (int k = 0; k < kFwd2K; k++) {
          const int j = 64 * h + (r >> 1);
          const double v = (j < n && k < n) ? scale * Vinv[2 * ((size_t)j * n + k) + (r & 1)] : 0.0;
          const size_t e = ((size_t)h * kM + r) * kFwd2K + k;
          split_host(v, fwd_hi[e], fwd_lo[e]);
        }
    for (int h = 0; h < 2; h++)
      for (int k = 0; k < kM; k++)
        for (int kk = 0; kk < kInv2K; kk++) {
          const int j = 64 * h + (kk >> 1), q = kk & 1;
          double v = 0.0;
          if (k < n && j < n) {
            const double vr = V[2 * ((size_t)k * n + j)], vi = V[2 * ((size_t)k * n + j) + 1];
            v = q == 0 ? vr : -vi;  // Re(V z) = Vr zr - Vi zi
          }
          const size_t e = ((size_t)h * kM + k) * kInv2K + kk;
          split_host(v, inv_hi[e], inv_lo[e]);
        }
    return;
  }
  for (int r = 0; r < kM; r++)
    for (int k = 0; k < kFwdK; k++) {
      double v = 0.0;
      const int j = r >> 1;
      if (j < n && k < n) v = scale * Vinv[2 * ((size_t)j * n + k) + (r & 1)];
      split_host(v, fwd_hi[r * kFwdK + k], fwd_lo[r * kFwdK + k]);
    }
  for (int r = 0; r < kM; r++)
    for (int kk = 0; kk < kInvK; kk++) {
      double v = 0.0;
      const int j = kk >> 1, q = kk & 1;
      const int k = r < 64 ? r : r - 64;
      if (k < n && j < n) {
        const double vr = V[2 * ((size_t)k * n + j)], vi = V[2 * ((size_t)k * n + j) + 1];
        if (r < 64) v = q == 0 ? vr : -vi;  // Re(V z) = Vr zr - Vi zi
        else v = q == 0 ? vi : vr;          // Im(V z) = Vi zr + Vr zi
      }
      split_host(v, inv_hi[r * kInvK + kk], inv_lo[r * kInvK + kk]);
    }
}

void launch_tc_forward(cudaStream_t s, int grid, int N, int n, View g, const void *f, bool f32,
                       const double *u0, const double *u0coef, const float *Ahi, const float *Alo,
                       double in_scale, int *errflag) {
  if (n > 64) {  // grid even: two CTAs (row halves) per tile
    if (f32)
      k_tc_forward<float, kFwd2K, kFwd2Nt, 2><<<grid, kTcThreads, kFwd2Smem, s>>>(
          N, n, g, static_cast<const float *>(f), u0, u0coef, Ahi, Alo, in_scale, errflag);
    else
      k_tc_forward<double, kFwd2K, kFwd2Nt, 2><<<grid, kTcThreads, kFwd2Smem, s>>>(
          N, n, g, static_cast<const double *>(f), u0, u0coef, Ahi, Alo, in_scale, errflag);
    return;
  }
  if (f32)
    k_tc_forward<float, kFwdK, kFwdNt, 1><<<grid, kTcThreads, kFwdSmem, s>>>(
        N, n, g, static_cast<const float *>(f), u0, u0coef, Ahi, Alo, in_scale, errflag);
  else
    k_tc_forward<double, kFwdK, kFwdNt, 1><<<grid, kTcThreads, kFwdSmem, s>>>(
        N, n, g, static_cast<const double *>(f), u0, u0coef, Ahi, Alo, in_scale, errflag);
}

void launch_tc_inverse(cudaStream_t s, int grid, int N, int n, double *u, View z0, View z1,
                       const int *final_buf, const float *Ahi, const float *Alo, float dscale,
                       bool accumulate, bool imag_check, unsigned long long *imag_bits, int *errflag) {
  if (n > 64) {
    k_tc_inverse2<<<grid, kTcThreads, kInv2Smem, s>>>(N, n, u, z0, z1, final_buf, Ahi, Alo, dscale,
                                                          accumulate ? 1 : 0, errflag);
    return;
  }
  k_tc_inverse<<<grid, kTcThreads, kInvSmem, s>>>(N, n, u, z0, z1, final_buf, Ahi, Alo, dscale,
                                                  accumulate ? 1 : 0, imag_check ? 1 : 0, imag_bits,
                                                  errflag);
}

}  // namespace pd
