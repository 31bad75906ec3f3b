// Time-direction transforms of eq. (1) on the 5th-generation tensor cores (tcgen05), for
// n <= 128 shifts.  Both are real GEMMs D[128 x Nt] = A[128 x K] B[K x Nt] over tiles of Nt
// grid points of one grid row, in TF32 with the 3-product split
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,  x_hi = x rounded to TF32, x_lo = x - x_hi,
// accumulated in FP32 in tensor memory: about 2^-21 relative per product, the
// FP32-compensated product the refinement needs because V can be ill-conditioned.
//
//   forward:  K = 64 (k < n),  rows 2j / 2j+1 of A = Re / Im of h^2 V^{-1}[j][k],
//             B[k][p] = fhat_k at point p (FP64 or FP32 input, rounded to FP32 then split);
//             g_j(p) = (D[2j][p], D[2j+1][p]).  For n > 64, K = 128 and two CTAs take
//             the shifts 0..63 and 64..127 of a tile.
//   inverse:  K = 128 (2j + re/im), row k of A = (Re V[k][j], -Im V[k][j]) and row 64 + k =
//             (Im V[k][j], Re V[k][j]), B[2j+q][p] = component q of z_j(p);
//             u_k(p) (+)= D[k][p], max |D[64+k][p]| is the imaginary-part check.  For n > 64
//             the rows are the 128 time steps (real part only) and K = 2n is split over the
//             two CTAs of a cluster.
//
// Operands live in shared memory in the K-major layout with 128-byte swizzling (8-row x
// 128-byte atoms, 16-byte chunk c of row r stored at chunk c ^ (r mod 8)); A is loaded
// once per CTA, B is built per tile by all threads from inputs that cp.async brought into
// a shared-memory stage one tile ahead.  One thread issues the MMAs and commits them to an
// mbarrier; two accumulators in tensor memory let the epilogue of one tile (tcgen05.ld
// through a padded shared-memory stage, so that the global stores are coalesced) run while
// the MMAs of the next one do.
#include "cplx.cuh"
#include "fpbits.cuh"
#include "pd_internal.h"
#include "tma.cuh"

#include <algorithm>

namespace pd {
namespace {

constexpr int kTcThreads = 512;
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

// D (+)= A B, kind::tf32: A in tensor memory (lane = row of A, one TF32 element per column),
// B in shared memory (descriptor)
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
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

// stores 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
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

// A (row-major [128][K] floats in global memory) into tensor memory at column col0: lane r
// holds row r, one element per column; warps 0-3 (lanes 32w..32w+31) store it
template <int K>
__device__ void load_a_tmem(const float *__restrict__ src, uint32_t tmem, int col0) {
  const int warp = (int)threadIdx.x >> 5, row = (int)threadIdx.x;
  if (warp < 4) {
#pragma unroll 1
    for (int c = 0; c < K / 32; c++) {
      float v[32];
      const float4 *p = reinterpret_cast<const float4 *>(src + (size_t)row * K + 32 * c);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const float4 x = p[q];
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
      }
      tmem_st32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(col0 + 32 * c), v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
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

// issues the 3 x (K/8) MMAs of one tile and commits them to `bar` (one thread); A hi/lo in
// tensor memory at columns a_hi, a_lo (8 columns per K step), B hi/lo in shared memory
template <int K, int NT>
__device__ __forceinline__ void issue_tile(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                           uint32_t b_lo, uint64_t *bar) {
  constexpr uint32_t idesc = idesc_tf32(kM, NT);
  uint32_t acc = 0;
#pragma unroll
  for (int ks = 0; ks < K / 8; ks++) {
    const uint32_t bo = (uint32_t)((ks >> 2) * NT * 128 + (ks & 3) * 32);
    mma_tf32_ta(d_tmem, a_hi + 8u * ks, desc_sw128(b_hi + bo), idesc, acc);
    acc = 1;
    mma_tf32_ta(d_tmem, a_hi + 8u * ks, desc_sw128(b_lo + bo), idesc, 1);
    mma_tf32_ta(d_tmem, a_lo + 8u * ks, desc_sw128(b_hi + bo), idesc, 1);
  }
  mma_commit(bar);
}

constexpr int kFwdK = 64, kFwdNt = 128;   // forward, n <= 64
constexpr int kFwd2K = 128, kFwd2Nt = 64;  // forward, 64 < n <= 128 (two CTAs per tile)
constexpr int kInvK = 128, kInvNt = 64;    // inverse, n <= 64
constexpr int kInv2K = 128, kInv2Nt = 64;  // inverse, 64 < n <= 128 (two-CTA cluster)
// forward epilogue: the accumulator's columns in passes of up to 64 (two chunks of 32, read by
// 8 warps at once); stage of 64 j rows x the pass's complex points, row stride 2 cols + 2
template <int NT> __host__ __device__ constexpr int fwd_pass_cols() { return NT < 64 ? NT : 64; }
template <int NT> __host__ __device__ constexpr int fwd_stage_bytes() { return 64 * (2 * fwd_pass_cols<NT>() + 2) * 4; }
// tensor memory: A hi at column 0, A lo at column K, the two accumulators from column 2K
constexpr int kTmemCols = 512;
static_assert(2 * 128 + 2 * 64 <= kTmemCols && 2 * 64 + 2 * 128 <= kTmemCols, "tensor memory");

// shared memory of the forward: B hi/lo, epilogue stage, input stage [K][NT] of the input
// type and the initial values of the tile's points, alignment slack
template <int K, int NT, typename InT> constexpr int fwd_smem() {
  return 2 * NT * K * 4 + fwd_stage_bytes<NT>() + NT * K * (int)sizeof(InT) + NT * 8 + 1024;
}
// the inverse: B hi/lo, stage [rows][NT + 4] (rows: 128, or 2 tile parities x 2 sources x 64
// in the cluster form; the row stride keeps 16-byte stores aligned and free of bank
// conflicts), z stage [64 shifts][NT] complex, u stage [64 rows][NT], slack
constexpr int kInvSmem = 2 * kInvNt * kInvK * 4 + kM * (kInvNt + 4) * 4 + 64 * kInvNt * 8 + 64 * kInvNt * 8 + 1024;
constexpr int kInv2Smem =
    2 * kInv2Nt * kInv2K * 4 + 2 * 2 * 64 * (kInv2Nt + 4) * 4 + 64 * kInv2Nt * 8 + 64 * kInv2Nt * 8 + 1024;
// the opt-in limit per block less the kernels' static shared memory
constexpr int kSmemLimit = 227 * 1024 - 1024;
static_assert(fwd_smem<kFwdK, kFwdNt, double>() <= kSmemLimit, "forward (n <= 64) exceeds shared memory");
static_assert(fwd_smem<kFwd2K, kFwd2Nt, double>() <= kSmemLimit, "forward (n > 64) exceeds shared memory");
static_assert(kInvSmem <= kSmemLimit, "inverse (n <= 64) exceeds shared memory");
static_assert(kInv2Smem <= kSmemLimit, "inverse (n > 64) exceeds shared memory");

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
  return p + ((1024 - (smem_u32(p) & 1023)) & 1023);
}

// g_j(p) = h^2 sum_k V^{-1}[j][k] fhat_k(p), fhat_k = in_scale (f_k + u0coef[k] u0), for the
// points p = (i, c0..c0+NT-1) of grid row i; written into the h^2-scaled level-0 RHS view
// (in_scale: a power of two that brings the refinement's FP64 residual near unit size).
// The rows of A are (Re, Im) of 64 shifts: with HALVES = 2 (n <= 128, K = 128) CTA x takes
// the shifts 64 (x mod 2) .. + 63, its A the matching half of the operand, and the tiles
// x / 2, x / 2 + gridDim.x / 2, ... (the two CTAs of a tile read its input once from DRAM).
// Pipeline: the input of tile t + 1 is copied into a shared-memory stage by cp.async
// (no registers hold it) and the accumulator of tile t - 1 is drained from the second
// accumulator in tensor memory while the MMAs of tile t run.  FP64 inputs become FP32 by
// bit operations (no FP64-pipe conversion per element).
template <typename InT, int K, int NT, int HALVES>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_forward(int N, int n, View g, const InT *__restrict__ f, const double *__restrict__ u0,
             const double *__restrict__ u0coef, const float *__restrict__ Ahi,
             const float *__restrict__ Alo, double in_scale, int *__restrict__ errflag) {
  constexpr int kB = NT * K * 4;
  constexpr int kItems = NT * (K / 4) / kTcThreads;  // (point, 4 consecutive k) items per thread
  constexpr int kCopies = NT * K / kTcThreads;       // input elements copied per thread
  static_assert(kItems * 4 <= 32, "the item masks hold 32 bits");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = align1024(smem_raw);
  unsigned char *sBhi = sm, *sBlo = sm + kB;
  float *S = reinterpret_cast<float *>(sBlo + kB);
  InT *stage = reinterpret_cast<InT *>(reinterpret_cast<unsigned char *>(S) + fwd_stage_bytes<NT>());  // [K][NT]
  double *su0 = reinterpret_cast<double *>(stage + NT * K);                           // [NT]
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = (int)blockIdx.x % HALVES, jbase = 64 * half;
  const int t0 = (int)blockIdx.x / HALVES, tstep = (int)gridDim.x / HALVES;
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  load_a_tmem<K>(Ahi + (size_t)half * kM * K, tmem, 0);
  load_a_tmem<K>(Alo + (size_t)half * kM * K, tmem, K);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t acc0 = tmem + 2 * K;  // first accumulator column
  const long long m = (long long)N * N;
  const int tpr = (int)((g.pitch + NT - 1) / NT);  // tiles per grid row
  const int total = N * tpr;
  const int nj = min(64, n - jbase);  // shifts of this CTA
  // which of a thread's item time steps carry the initial-value term (u0coef[k] != 0,
  // tested on the bits): the same in every tile
  unsigned cmask = 0;
  if (u0)
    for (int q = 0; q < kItems; q++)
      for (int e = 0; e < 4; e++) {
        const int k = 4 * ((tid + q * kTcThreads) / NT) + e;
        if (k < n && (__double_as_longlong(u0coef[k]) << 1) != 0) cmask |= 1u << (4 * q + e);
      }
  const int s_in = pow2_exponent(in_scale);
  const float fs_in = __uint_as_float((unsigned)(s_in + 127) << 23);  // FP32 inputs: |s_in| < 127
  // copies of tile t into the stage (element (k, p) of the tile) and of its initial values
  // where the term is used.  Elements outside the grid or with k >= n are not copied: the
  // rows k >= n keep the zeros written below (A is zero there too), the columns beyond the
  // grid produce outputs that are not stored (each output column depends on its own B
  // column only)
  auto fetch = [&](int t) {
    const int i = t / tpr, c0 = (t % tpr) * NT;
    const uint32_t sbase = smem_u32(stage);
#pragma unroll
    for (int e = 0; e < kCopies; e++) {
      const int q = tid + e * kTcThreads, k = q / NT, p = q % NT;
      if (k < n && c0 + p < N)
        cpa(sbase + (uint32_t)(q * (int)sizeof(InT)), f + (long long)k * m + (long long)i * N + c0 + p,
            (int)sizeof(InT), true);
    }
    if (u0 && tid < NT && c0 + tid < N) cpa(smem_u32(su0 + tid), u0 + (long long)i * N + c0 + tid, 8, true);
    cpa_commit();
  };
  for (int q = tid; q < NT * K; q += kTcThreads) stage[q] = (InT)0;
  for (int q = tid; q < NT; q += kTcThreads) su0[q] = 0.0;
  __syncthreads();
  auto to_op = [&](InT v) -> float {
    if constexpr (sizeof(InT) == 8) return f64_to_f32(v, s_in);
    else return v * fs_in;
  };
  // g of tile t from accumulator buf, PC columns a pass: warp w < PC / 8 reads the lanes
  // 32 (w mod 4) .. (rows 2j+q of D) of the 32 columns 32 (w / 4) .. of the pass; the stage
  // makes the stores coalesced
  constexpr int PC = fwd_pass_cols<NT>(), SRF = 2 * PC + 2;
  static_assert(4 * (PC / 32) <= kTcThreads / 32, "one warp per lane group and column chunk");
  auto epilogue = [&](int t, int buf) {
    const int i = t / tpr, c0 = (t % tpr) * NT;
    for (int pass = 0; pass < NT / PC; pass++) {
      if (warp < 4 * (PC / 32)) {
        float v[32];
        const int chunk = warp >> 2, row = 32 * (warp & 3) + lane, j = row >> 1, q = row & 1;
        tmem_ld32(acc0 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(buf * NT + PC * pass + 32 * chunk), v);
        if (j < nj)
#pragma unroll
          for (int cc = 0; cc < 32; cc++) S[j * SRF + 2 * (32 * chunk + cc) + q] = v[cc];
      }
      __syncthreads();
      for (int it = tid; it < nj * PC; it += kTcThreads) {
        const int j = it / PC, cc = it % PC;
        const int c = c0 + PC * pass + cc;
        if (c < N) {
          const float2 val = *reinterpret_cast<const float2 *>(&S[j * SRF + 2 * cc]);
          reinterpret_cast<float2 *>(g.p)[(jbase + j) * g.plane + (long long)i * g.pitch + c] = val;
        }
      }
      __syncthreads();
    }
  };
  bool ok = true;
  int idx = 0, tprev = 0;
  int t = t0;
  if (t < total) fetch(t);
  for (; t < total; t += tstep, idx++) {
    bool w = true;
    if (idx > 0) w = mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));  // B free
    cpa_wait<0>();                                                          // stage full
    if (!__syncthreads_and(w)) {
      ok = false;
      break;
    }
    tc_fence_after();
    // B[p][k] = fhat_k(i, c0 + p), split into TF32 hi/lo, 16-byte swizzled chunks
#pragma unroll
    for (int q = 0; q < kItems; q++) {
      const int it = tid + q * kTcThreads;
      const int p = it % NT, kq = it / NT;
      float x[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const InT v = stage[(4 * kq + e) * NT + p];
        x[e] = (cmask >> (4 * q + e) & 1u)
                   ? f64_to_f32(((double)v + u0coef[4 * kq + e] * su0[p]) * in_scale)
                   : to_op(v);
      }
      float4 hi, lo;
      split_tf32(x[0], hi.x, lo.x);
      split_tf32(x[1], hi.y, lo.y);
      split_tf32(x[2], hi.z, lo.z);
      split_tf32(x[3], hi.w, lo.w);
      *reinterpret_cast<float4 *>(sBhi + sw_off(p, kq, NT)) = hi;
      *reinterpret_cast<float4 *>(sBlo + sw_off(p, kq, NT)) = lo;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();  // B complete, the stage free
    if (tid == 0) {
      tc_fence_after();
      issue_tile<K, NT>(acc0 + (uint32_t)((idx & 1) * NT), tmem, tmem + K, smem_u32(sBhi), smem_u32(sBlo),
                        &bar);
    }
    if (t + tstep < total) fetch(t + tstep);
    if (idx > 0) epilogue(tprev, (idx - 1) & 1);
    tc_fence_before();
    tprev = t;
  }
  if (ok && idx > 0) {
    const bool w = mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));
    if (__syncthreads_and(w)) {
      tc_fence_after();
      epilogue(tprev, (idx - 1) & 1);
    } else {
      ok = false;
    }
  }
  cpa_wait<0>();
  if (!ok && tid == 0) {
    atomicOr(errflag, 4);
    mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));  // let the MMAs in flight finish
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// copies of the z values of 64 shifts (jbase ..) at the NT points of a tile into the
// stage [64][NT] (complex, from z1 where final_buf is set).  Shifts j >= n and points
// beyond the grid are not copied: the rows j >= n keep the zeros the kernel writes first
// (V is zero there too), the columns beyond the grid give outputs that are not stored.
// zsel: bit e set where the thread's e-th copy reads z1 (z1_select, the same in every tile)
template <int NT>
__device__ __forceinline__ unsigned z1_select(const int *final_buf, int n, int jbase) {
  unsigned m = 0;
  if (final_buf)
    for (int e = 0; e < 64 * NT / kTcThreads; e++) {
      const int jj = jbase + ((int)threadIdx.x + e * kTcThreads) / NT;
      if (jj < n && final_buf[jj]) m |= 1u << e;
    }
  return m;
}
template <int NT>
__device__ __forceinline__ void copy_z(const View &z0, const View &z1, unsigned zsel, int n, int N,
                                       int jbase, int i, int c0, uint32_t sbase) {
  static_assert(64 * NT / kTcThreads <= 32, "the selection mask holds 32 bits");
#pragma unroll
  for (int e = 0; e < 64 * NT / kTcThreads; e++) {
    const int q = (int)threadIdx.x + e * kTcThreads, jl = q / NT, p = q % NT, jj = jbase + jl;
    if (jj < n && c0 + p < N) {
      const bool use1 = (zsel >> e) & 1u;
      const float2 *zp = reinterpret_cast<const float2 *>(use1 ? z1.p : z0.p);
      const long long plane = use1 ? z1.plane : z0.plane, pitch = use1 ? z1.pitch : z0.pitch;
      cpa(sbase + (uint32_t)(q * 8), zp + jj * plane + (long long)i * pitch + c0 + p, 8, true);
    }
  }
}
// copies of u at rows kbase .. kbase + 63 (< n) and the NT points of a tile into [64][NT]
// (only the entries that exist: the others are not read); thread tid copies the elements
// it later reads (it = tid + e * threads)
template <int NT>
__device__ __forceinline__ void copy_u(const double *u, int n, int N, long long m, int kbase, int i, int c0,
                                       uint32_t sbase) {
#pragma unroll
  for (int e = 0; e < 64 * NT / kTcThreads; e++) {
    const int q = (int)threadIdx.x + e * kTcThreads, k = kbase + q / NT, c = c0 + q % NT;
    if (k < n && c < N) cpa(sbase + (uint32_t)(q * 8), u + (long long)k * m + (long long)i * N + c, 8, true);
  }
}

// B of the inverse from the z stage: B[p][2 jl + q] = component q of z_jl(p), TF32 split
template <int NT>
__device__ __forceinline__ void build_b_inv(const float2 *zst, unsigned char *sBhi, unsigned char *sBlo) {
#pragma unroll
  for (int q = 0; q < NT * 32 / kTcThreads; q++) {
    const int it = (int)threadIdx.x + q * kTcThreads;
    const int p = it % NT, qq = it / NT;
    const float2 a = zst[(2 * qq) * NT + p], b = zst[(2 * qq + 1) * NT + p];
    float4 hi, lo;
    split_tf32(a.x, hi.x, lo.x);
    split_tf32(a.y, hi.y, lo.y);
    split_tf32(b.x, hi.z, lo.z);
    split_tf32(b.y, hi.w, lo.w);
    *reinterpret_cast<float4 *>(sBhi + sw_off(p, qq, NT)) = hi;
    *reinterpret_cast<float4 *>(sBlo + sw_off(p, qq, NT)) = lo;
  }
}

// u_k(p) (+)= dscale Re sum_j V[k][j] z_j(p) for p = (i, c0..c0+NT-1); z_j is read from
// z1 where final_buf[j] is set, else from z0; imag_check: atomic max of |Im| (bits of a
// double).  The forward's pipeline: z of tile t + 1 and the u values tile t accumulates
// into arrive in shared-memory stages by cp.async while the MMAs of tile t run and u of
// tile t - 1 is written from the other accumulator.  FP32 -> FP64 by bit operations; one
// FP64 add per output when accumulating.
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_inverse(int N, int n, double *__restrict__ u, View z0, View z1, const int *__restrict__ final_buf,
             const float *__restrict__ Ahi, const float *__restrict__ Alo, float dscale, int accumulate,
             int imag_check, unsigned long long *imag_bits, int *__restrict__ errflag) {
  constexpr int NT = kInvNt, K = kInvK, SR = NT + 4;
  constexpr int kB = NT * K * 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = align1024(smem_raw);
  unsigned char *sBhi = sm, *sBlo = sm + kB;
  float *S = reinterpret_cast<float *>(sBlo + kB);                   // [128][NT + 4]
  float2 *zst = reinterpret_cast<float2 *>(S + kM * SR);             // [64][NT]
  double *ust = reinterpret_cast<double *>(zst + 64 * NT);           // [64][NT]
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float red[kTcThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  load_a_tmem<K>(Ahi, tmem, 0);
  load_a_tmem<K>(Alo, tmem, K);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t acc0 = tmem + 2 * K;
  for (int q = tid; q < 64 * NT; q += kTcThreads) zst[q] = make_float2(0.f, 0.f);
  const unsigned zsel = z1_select<NT>(final_buf, n, 0);
  __syncthreads();
  const long long m = (long long)N * N;
  const int tpr = (int)((z0.pitch + NT - 1) / NT);
  const int total = N * tpr;
  float imax = 0.f;
  constexpr int kAcc = 64 * NT / kTcThreads;  // u values of a tile per thread (rows k < 64)
  auto epilogue = [&](int t, int buf) {
    const int i = t / tpr, c0 = (t % tpr) * NT;
    if (warp < 4 * (NT / 32)) {  // warps w and w + 4 read the same lanes, columns 32 (w / 4) ..
      float v[32];
      const int chunk = warp >> 2, row = 32 * (warp & 3) + lane;
      tmem_ld32(acc0 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(buf * NT + 32 * chunk), v);
#pragma unroll
      for (int cc = 0; cc < 32; cc += 4)
        *reinterpret_cast<float4 *>(&S[row * SR + 32 * chunk + cc]) = make_float4(v[cc], v[cc + 1], v[cc + 2], v[cc + 3]);
    }
    if (accumulate) cpa_wait<1>();  // this thread's u copies of tile t (the z copies of t + 2 may pend)
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kAcc; q++) {
      const int it = tid + q * kTcThreads;
      const int k = it / NT, cc = it % NT, c = c0 + cc;
      if (k < n && c < N) {
        const double d = f32_to_f64(S[k * SR + cc] * dscale);
        u[(long long)k * m + (long long)i * N + c] = accumulate ? ust[it] + d : d;
        if (imag_check) imax = fmaxf(imax, fabsf(S[(64 + k) * SR + cc] * dscale));
      }
    }
    __syncthreads();
  };
  bool ok = true;
  int idx = 0, tprev = 0;
  int t = blockIdx.x;
  if (t < total) {
    copy_z<NT>(z0, z1, zsel, n, N, 0, t / tpr, (t % tpr) * NT, smem_u32(zst));
    cpa_commit();
  }
  for (; t < total; t += gridDim.x, idx++) {
    bool w = true;
    if (idx > 0) w = mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));
    if (accumulate && idx > 0) cpa_wait<1>();  // z of tile t (the u copies of tprev may pend)
    else cpa_wait<0>();
    if (!__syncthreads_and(w)) {
      ok = false;
      break;
    }
    tc_fence_after();
    build_b_inv<NT>(zst, sBhi, sBlo);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_tile<K, NT>(acc0 + (uint32_t)((idx & 1) * NT), tmem, tmem + K, smem_u32(sBhi), smem_u32(sBlo),
                        &bar);
    }
    const int tn = t + (int)gridDim.x;
    if (tn < total) copy_z<NT>(z0, z1, zsel, n, N, 0, tn / tpr, (tn % tpr) * NT, smem_u32(zst));
    cpa_commit();
    if (idx > 0) epilogue(tprev, (idx - 1) & 1);
    if (accumulate) {
      copy_u<NT>(u, n, N, m, 0, t / tpr, (t % tpr) * NT, smem_u32(ust));
      cpa_commit();
    }
    tc_fence_before();
    tprev = t;
  }
  if (ok && idx > 0) {
    const bool w = mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));
    if (__syncthreads_and(w)) {
      tc_fence_after();
      if (accumulate) cpa_wait<0>();
      epilogue(tprev, (idx - 1) & 1);
    } else {
      ok = false;
    }
  }
  cpa_wait<0>();
  if (!ok && tid == 0) {
    atomicOr(errflag, 4);
    mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));
  }
  if (imag_check) {
    for (int o = 16; o > 0; o >>= 1) imax = fmaxf(imax, __shfl_down_sync(0xffffffffu, imax, o));
    if (lane == 0) red[warp] = imax;
  }
  tc_fence_before();
  __syncthreads();
  if (imag_check && tid == 0) {
    float mx = 0.f;
    for (int w = 0; w < kTcThreads / 32; w++) mx = fmaxf(mx, red[w]);
    atomicMax(imag_bits, (unsigned long long)__double_as_longlong(f32_to_f64(mx)));
  }
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
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
// 16 bytes into the shared memory of a CTA of the cluster (addr 16-byte aligned)
__device__ __forceinline__ void st_cluster4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// u_k(p) (+)= dscale Re sum_j V[k][j] z_j(p) for k < 128 and the points p = (i, c0..c0+31):
// CTA r of a cluster of two multiplies the shifts j = 64 r .. 64 r + 63 (its half of K,
// A = its half of the operand) into D_r[128 x 32]; CTA r owns the rows k = 64 r .. 64 r + 63
// of u: it keeps those rows of D_r and stores the other half into its peer's stage through
// distributed shared memory; after a cluster barrier it writes u_k = D_0[k] + D_1[k] for its
// own rows (the stage slot alternates with the tile parity, which is also the accumulator's).
// The imaginary part is not formed on this route.  Both CTAs walk the same tiles and meet at every cluster
// barrier, also after a bounded wait ran out (then they only skip the work), so neither
// can wait for the other forever.  The pipeline is the one of k_tc_inverse.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTcThreads, 1)
k_tc_inverse2(int N, int n, double *__restrict__ u, View z0, View z1, const int *__restrict__ final_buf,
              const float *__restrict__ Ahi, const float *__restrict__ Alo, float dscale, int accumulate,
              int *__restrict__ errflag) {
  constexpr int NT = kInv2Nt, K = kInv2K, SR = NT + 4;
  constexpr int kB = NT * K * 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = align1024(smem_raw);
  unsigned char *sBhi = sm, *sBlo = sm + kB;
  float *S = reinterpret_cast<float *>(sBlo + kB);          // [2 parities][2 sources][64][NT + 4]
  float2 *zst = reinterpret_cast<float2 *>(S + 4 * 64 * SR);  // [64][NT]
  double *ust = reinterpret_cast<double *>(zst + 64 * NT);   // [64][NT]
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const int jbase = 64 * (int)rank, kbase = 64 * (int)rank;
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  load_a_tmem<K>(Ahi + (size_t)rank * kM * K, tmem, 0);
  load_a_tmem<K>(Alo + (size_t)rank * kM * K, tmem, K);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t acc0 = tmem + 2 * K;
  for (int q = tid; q < 64 * NT; q += kTcThreads) zst[q] = make_float2(0.f, 0.f);
  const unsigned zsel = z1_select<NT>(final_buf, n, jbase);
  __syncthreads();
  const uint32_t S_peer = peer_addr(smem_u32(S), rank ^ 1u);
  const long long m = (long long)N * N;
  const int tpr = (int)((z0.pitch + NT - 1) / NT);
  const int total = N * tpr;
  const int t0 = (int)blockIdx.x / 2, tstep = (int)gridDim.x / 2;
  constexpr int kAcc = 64 * NT / kTcThreads;  // own u values of a tile per thread
  bool ok = true;
  // the stage of tile parity sb: own partial rows at [sb][0], the peer's at [sb][1]; one slot
  // per parity, so one cluster barrier per tile orders both the stores and the reuse (the
  // peer writes slot sb again two tiles later, after passing the next barrier, which this
  // CTA reaches only when it has read slot sb)
  auto epilogue = [&](int t, int buf) {
    const int i = t / tpr, c0 = (t % tpr) * NT;
    float *Sb = S + buf * 2 * 64 * SR;
    if (ok && warp < 4 * (NT / 32)) {  // warps w and w + 4 read the same lanes, columns 32 (w / 4) ..
      float v[32];
      const int chunk = warp >> 2, row = 32 * (warp & 3) + lane, r64 = row & 63;
      tmem_ld32(acc0 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(buf * NT + 32 * chunk), v);
      if ((row >> 6) == (int)rank) {
#pragma unroll
        for (int cc = 0; cc < 32; cc += 4)
          *reinterpret_cast<float4 *>(&Sb[r64 * SR + 32 * chunk + cc]) = make_float4(v[cc], v[cc + 1], v[cc + 2], v[cc + 3]);
      } else {
        const uint32_t base = S_peer + (uint32_t)(((buf * 2 * 64 + 64 + r64) * SR + 32 * chunk) * 4);
#pragma unroll
        for (int cc = 0; cc < 32; cc += 4) st_cluster4(base + 4u * cc, v[cc], v[cc + 1], v[cc + 2], v[cc + 3]);
      }
    }
    if (accumulate) cpa_wait<1>();
    cluster_sync();  // both partials of this CTA's rows are in its stage
    if (ok) {
#pragma unroll
      for (int q = 0; q < kAcc; q++) {
        const int it = tid + q * kTcThreads;
        const int r64 = it / NT, cc = it % NT, k = kbase + r64, c = c0 + cc;
        if (k < n && c < N) {
          const double d = f32_to_f64((Sb[r64 * SR + cc] + Sb[(64 + r64) * SR + cc]) * dscale);
          u[(long long)k * m + (long long)i * N + c] = accumulate ? ust[it] + d : d;
        }
      }
    }
  };
  int idx = 0, tprev = 0, fail_par = 0;
  int t = t0;
  if (t < total) {
    copy_z<NT>(z0, z1, zsel, n, N, jbase, t / tpr, (t % tpr) * NT, smem_u32(zst));
    cpa_commit();
  }
  for (; t < total; t += tstep, idx++) {
    if (idx > 0 && ok) {
      const bool w = mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));
      ok = __syncthreads_and(w);
      fail_par = (idx - 1) & 1;
    }
    if (accumulate && idx > 0) cpa_wait<1>();
    else cpa_wait<0>();
    __syncthreads();
    tc_fence_after();
    if (ok) {
      build_b_inv<NT>(zst, sBhi, sBlo);
      fence_proxy_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    if (ok && tid == 0) {
      tc_fence_after();
      issue_tile<K, NT>(acc0 + (uint32_t)((idx & 1) * NT), tmem, tmem + K, smem_u32(sBhi), smem_u32(sBlo),
                        &bar);
    }
    const int tn = t + tstep;
    if (tn < total) copy_z<NT>(z0, z1, zsel, n, N, jbase, tn / tpr, (tn % tpr) * NT, smem_u32(zst));
    cpa_commit();
    if (idx > 0) epilogue(tprev, (idx - 1) & 1);
    if (accumulate) {
      copy_u<NT>(u, n, N, m, kbase, t / tpr, (t % tpr) * NT, smem_u32(ust));
      cpa_commit();
    }
    tc_fence_before();
    tprev = t;
  }
  if (idx > 0) {
    if (ok) {
      const bool w = mbar_wait_bounded(&bar, (uint32_t)((idx - 1) & 1));
      ok = __syncthreads_and(w);
      fail_par = (idx - 1) & 1;
    }
    tc_fence_after();
    if (accumulate) cpa_wait<0>();
    epilogue(tprev, (idx - 1) & 1);
  }
  cpa_wait<0>();
  if (!ok && tid == 0) {
    atomicOr(errflag, 4);
    mbar_wait_bounded(&bar, (uint32_t)fail_par);  // let the MMAs in flight finish
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
  cluster_sync();  // no CTA leaves while its peer may still address its shared memory
}

}  // namespace

bool tc_transforms_supported(int N, int n) { return n <= 128 && N >= 127; }

cudaError_t prepare_tc_transforms() {
  cudaError_t e;
#define PD_TC_ATTR(K_, S_)                                                         \
  e = cudaFuncSetAttribute(K_, cudaFuncAttributeMaxDynamicSharedMemorySize, S_); \
  if (e != cudaSuccess) return e;
  PD_TC_ATTR((k_tc_forward<double, kFwdK, kFwdNt, 1>), (fwd_smem<kFwdK, kFwdNt, double>()))
  PD_TC_ATTR((k_tc_forward<float, kFwdK, kFwdNt, 1>), (fwd_smem<kFwdK, kFwdNt, float>()))
  PD_TC_ATTR((k_tc_forward<double, kFwd2K, kFwd2Nt, 2>), (fwd_smem<kFwd2K, kFwd2Nt, double>()))
  PD_TC_ATTR((k_tc_forward<float, kFwd2K, kFwd2Nt, 2>), (fwd_smem<kFwd2K, kFwd2Nt, float>()))
  PD_TC_ATTR(k_tc_inverse, kInvSmem)
  PD_TC_ATTR(k_tc_inverse2, kInv2Smem)
#undef PD_TC_ATTR
  return cudaSuccess;
}

// A operands (host): TF32 splits of the scaled forward matrix and of the inverse matrix
// in the row layouts described at the top of this file.
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
      k_tc_forward<float, kFwd2K, kFwd2Nt, 2><<<grid, kTcThreads, fwd_smem<kFwd2K, kFwd2Nt, float>(), s>>>(
          N, n, g, static_cast<const float *>(f), u0, u0coef, Ahi, Alo, in_scale, errflag);
    else
      k_tc_forward<double, kFwd2K, kFwd2Nt, 2><<<grid, kTcThreads, fwd_smem<kFwd2K, kFwd2Nt, double>(), s>>>(
          N, n, g, static_cast<const double *>(f), u0, u0coef, Ahi, Alo, in_scale, errflag);
    return;
  }
  if (f32)
    k_tc_forward<float, kFwdK, kFwdNt, 1><<<grid, kTcThreads, fwd_smem<kFwdK, kFwdNt, float>(), s>>>(
        N, n, g, static_cast<const float *>(f), u0, u0coef, Ahi, Alo, in_scale, errflag);
  else
    k_tc_forward<double, kFwdK, kFwdNt, 1><<<grid, kTcThreads, fwd_smem<kFwdK, kFwdNt, double>(), s>>>(
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
