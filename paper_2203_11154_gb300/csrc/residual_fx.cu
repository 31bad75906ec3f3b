// Residual of the shifted systems of eq. (2) for the refined solves without FP64
// instructions (GB300 issues FP64 at 1/58 of its FP32 rate; measured 1.26 vs 73 TFLOP/s),
// with the arithmetic of the refinement residual of eq. (1) (residual_ws.cu):
//
//   - Fixed point: the values of a halo tile are truncated to units of 2^-S, one scale per
//     tile and complex component, S = 1081 - (largest biased exponent in the tile), so
//     every |value| < 2^59 units; the truncation, below 2^-58 max|z| of the tile, is under
//     the FP64 rounding of the largest value.  A value v is held as three FP32 limbs
//     t2 2^42 + t1 2^21 + t0 (|t2| < 2^17, t1, t0 < 2^21, all of the value's sign), each an
//     exact FP32 number (ff::to_limbs).
//   - The stencil difference T1 = 4 z - (sum of neighbours), the cancellation-critical
//     part, is exact: per limb, 4 c - (sum of 4 neighbours) is an integer multiple of the
//     limb unit below 2^24 units, exact in FP32 arithmetic (FMA pipe, no integer work).
//   - The remaining arithmetic is float-float (pairs hi + lo of FP32) with the error-free
//     transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA product split.
//   - FP64 inputs become float-float by bit operations: hi = the value truncated to 24
//     significant bits, lo = the remaining 29 bits converted to FP32.
#include <cstdint>

#include "ff.cuh"
#include "pd_internal.h"

namespace pd {
namespace {

using namespace ff;

constexpr int kRxRows = 16, kRxCols = 128, kRxThreads = 256;
constexpr int kRxHR = kRxRows + 2, kRxHC = kRxCols + 2;  // halo tile
constexpr int kRxHalo = kRxHR * kRxHC;
constexpr int kRxPer = (kRxHalo + kRxThreads - 1) / kRxThreads;  // halo values per thread
constexpr int kRxPts = kRxRows * kRxCols / kRxThreads;           // rows per thread (8)
constexpr int kRxWarps = kRxThreads / 32;


__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------------------
// The residual of the shifted systems of eq. (2) for the refined solves, with the same
// arithmetic: r_j = b_j - lam_j z_j - (kappa/h^2)(4 z_j - sum of the 4 neighbours of z_j),
// complex, z_j and b_j in FP64; output in FP32 times oscale (the scaling of the level-0
// right-hand side) with the CTA's sum of |r|^2.  The stencil difference is exact per
// component (the real parts, then the imaginary parts of a halo tile go through the limb
// buffer, each with its own scale); lam_j z_j and the sums are float-float.  One shift per
// CTA row (grid (gx, n)), tiles of 16 x 128 points strided over blockIdx.x; frozen shifts
// get a zero right-hand side and no sums.

struct SxShared {
  ulonglong2 raw[2][kRxHalo];  // FP64 complex bits of the halo tile, double-buffered
  float4 limb[kRxHalo];        // limbs of one component
  unsigned red_e[2][kRxWarps];
  float2 redf[kRxWarps];
};
constexpr size_t kSxSmem = sizeof(SxShared);

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}

// the complex halo tile of z_j at (i0, c0) into raw: zero outside the grid
__device__ __forceinline__ void issue_halo_c(ulonglong2 *raw, const double2 *zj, int N, int i0, int c0) {
  const int lane = threadIdx.x & 31;
  const bool cols_in = c0 >= 1 && c0 + kRxCols < N;
  for (int hr = threadIdx.x >> 5; hr < kRxHR; hr += kRxWarps) {
    const int i = i0 - 1 + hr;
    ulonglong2 *dst = raw + hr * kRxHC + lane;
    if ((unsigned)i >= (unsigned)N) {
#pragma unroll
      for (int j = 0; j < 4; j++) cp_async16(dst + 32 * j, zj, 0);
      if (lane < kRxHC - 128) cp_async16(dst + 128, zj, 0);
      continue;
    }
    const double2 *src = zj + (long long)i * N + (c0 - 1) + lane;
    if (cols_in) {
#pragma unroll
      for (int j = 0; j < 4; j++) cp_async16(dst + 32 * j, src + 32 * j, 16);
      if (lane < kRxHC - 128) cp_async16(dst + 128, src + 128, 16);
    } else {
#pragma unroll
      for (int j = 0; j < 5; j++) {
        const int hc = lane + 32 * j;
        if (j < 4 || hc < kRxHC) {
          const bool in = (unsigned)(c0 - 1 + hc) < (unsigned)N;
          cp_async16(dst + 32 * j, in ? src + 32 * j : zj, in ? 16 : 0);
        }
      }
    }
  }
}

// the exact 4c - (sum of neighbours) of the thread's points for the limbs in sh.limb, as
// float-float pairs in units of the limbs' scale
__device__ __forceinline__ void stencil_limbs(const float4 *__restrict__ limb, int pc, int pr0, DF (&t1)[kRxPts]) {
  const float4 *L = limb + pc + 1;
  float4 up = L[pr0 * kRxHC], cu = L[(pr0 + 1) * kRxHC];
#pragma unroll
  for (int t = 0; t < kRxPts; t++) {
    const int hr = pr0 + t + 1;
    const float4 dn = L[(hr + 1) * kRxHC];
    const float4 lf = L[hr * kRxHC - 1], rt = L[hr * kRxHC + 1];
    const float a2 = __fmaf_rn(4.f, cu.x, -__fadd_rn(__fadd_rn(up.x, dn.x), __fadd_rn(lf.x, rt.x)));
    const float a1 = __fmaf_rn(4.f, cu.y, -__fadd_rn(__fadd_rn(up.y, dn.y), __fadd_rn(lf.y, rt.y)));
    const float a0 = __fmaf_rn(4.f, cu.z, -__fadd_rn(__fadd_rn(up.z, dn.z), __fadd_rn(lf.z, rt.z)));
    t1[t] = two_sum(a2, a1);
    t1[t].lo = __fadd_rn(t1[t].lo, a0);
    up = cu;
    cu = dn;
  }
}

__global__ void __launch_bounds__(kRxThreads, 2)
k_shift_residual_fx(int N, const double2 *__restrict__ z, const double2 *__restrict__ b,
                    const double2 *__restrict__ c1, double off, float oscale,
                    const float *__restrict__ sc, View out, const int *__restrict__ frozen,
                    double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned char sx_smem[];
  SxShared &sh = *reinterpret_cast<SxShared *>(sx_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j = blockIdx.y;
  const long long m = (long long)N * N;
  const int tx = (N + kRxCols - 1) / kRxCols;
  const int tiles = tx * ((N + kRxRows - 1) / kRxRows);
  const int pc = tid % kRxCols, pr0 = (tid / kRxCols) * kRxPts;
  float2 *o = reinterpret_cast<float2 *>(out.p) + (long long)j * out.plane;
  if (frozen && frozen[j]) {
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int i0 = (t / tx) * kRxRows, c = (t % tx) * kRxCols + pc;
#pragma unroll
      for (int q = 0; q < kRxPts; q++) {
        const int i = i0 + pr0 + q;
        if (i < N && c < N) o[(long long)i * out.pitch + c] = make_float2(0.f, 0.f);
      }
    }
    if (tid == 0) part[(long long)j * gridDim.x + blockIdx.x] = 0.0;
    return;
  }
  const double2 *zj = z + (long long)j * m, *bj = b + (long long)j * m;
  // lam_j = c1_j - 4 kappa/h^2 as float-float pairs; kappa/h^2
  const double2 cj = c1[j];
  const DF lr = split(cj.x - 4.0 * off), li = split(cj.y), offd = split(off);
  const float scj = sc[j];  // a power of two keeping the FP32 right-hand side near unit size
  DF ar = {0.f, 0.f};
  int t = blockIdx.x, buf = 0;
  if (t < tiles) issue_halo_c(sh.raw[0], zj, N, (t / tx) * kRxRows, (t % tx) * kRxCols);
  cp_async_commit();
  for (; t < tiles; t += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();  // raw[buf] complete; the previous tile is done with limb[]
    const int t2 = t + gridDim.x;
    if (t2 < tiles) issue_halo_c(sh.raw[buf ^ 1], zj, N, (t2 / tx) * kRxRows, (t2 % tx) * kRxCols);
    cp_async_commit();
    const int i0 = (t / tx) * kRxRows, c0 = (t % tx) * kRxCols, c = c0 + pc;
    const ulonglong2 *raw = sh.raw[buf];
    // 1. largest exponent of each component
    unsigned er = 0, ei = 0;
#pragma unroll
    for (int e = 0; e < kRxPer; e++) {
      const int q = tid + e * kRxThreads;
      if (q < kRxHalo) {
        const ulonglong2 v = raw[q];
        er = max(er, (unsigned)(v.x >> 32) & 0x7FFFFFFFu);
        ei = max(ei, (unsigned)(v.y >> 32) & 0x7FFFFFFFu);
      }
    }
    er = __reduce_max_sync(0xffffffffu, er) >> 20;
    ei = __reduce_max_sync(0xffffffffu, ei) >> 20;
    if (lane == 0) {
      sh.red_e[0][warp] = er;
      sh.red_e[1][warp] = ei;
    }
    __syncthreads();
    er = ei = 0;
#pragma unroll
    for (int w = 0; w < kRxWarps; w++) {
      er = max(er, sh.red_e[0][w]);
      ei = max(ei, sh.red_e[1][w]);
    }
    // 2. real parts: limbs, then the exact stencil difference
#pragma unroll
    for (int e = 0; e < kRxPer; e++) {
      const int q = tid + e * kRxThreads;
      if (q < kRxHalo) sh.limb[q] = to_limbs(raw[q].x, er);
    }
    __syncthreads();
    DF tr[kRxPts], ti[kRxPts];
    stencil_limbs(sh.limb, pc, pr0, tr);
    // the right-hand side of the thread's points, requested now for step 4
    const int nrow = c < N ? min(kRxPts, N - i0 - pr0) : 0;
    const long long x0 = (long long)(i0 + pr0) * N + c;
    double2 bq[kRxPts];
#pragma unroll
    for (int q = 0; q < kRxPts; q++) bq[q] = q < nrow ? bj[x0 + q * N] : make_double2(0.0, 0.0);
    __syncthreads();
    // 3. imaginary parts
#pragma unroll
    for (int e = 0; e < kRxPer; e++) {
      const int q = tid + e * kRxThreads;
      if (q < kRxHalo) sh.limb[q] = to_limbs(raw[q].y, ei);
    }
    __syncthreads();
    stencil_limbs(sh.limb, pc, pr0, ti);
    // 4. r = b - lam z - (kappa/h^2) T1 per point
    const bool bad = er > 1081 + 126 || ei > 1081 + 126;
    const int Sr = 1081 - (int)er, Si = 1081 - (int)ei;
    const DF qr = df_scale_down(offd, Sr > 252 ? 252 : Sr), qi = df_scale_down(offd, Si > 252 ? 252 : Si);
    float rowr = 0.f;
#pragma unroll
    for (int q = 0; q < kRxPts; q++) {
      if (q >= nrow) break;
      const ulonglong2 zc = raw[(pr0 + q + 1) * kRxHC + pc + 1];
      const DF zr = split_bits((uint32_t)(zc.x >> 32), (uint32_t)zc.x);
      const DF zi = split_bits((uint32_t)(zc.y >> 32), (uint32_t)zc.y);
      const DF br = split(bq[q].x), bi = split(bq[q].y);
      // real: br - lr zr + li zi - qr T1r; imaginary: bi - lr zi - li zr - qi T1i
      const DF p1 = df_mul_un(lr, zr), p2 = df_mul_un(li, zi), p3 = df_mul_un(qr, tr[q]);
      const DF p4 = df_mul_un(lr, zi), p5 = df_mul_un(li, zr), p6 = df_mul_un(qi, ti[q]);
      float lo = __fadd_rn(__fsub_rn(br.lo, p1.lo), __fsub_rn(p2.lo, p3.lo));
      DF s1 = two_sum(br.hi, -p1.hi);
      float el = s1.lo;
      s1 = two_sum(s1.hi, p2.hi);
      el = __fadd_rn(el, s1.lo);
      s1 = two_sum(s1.hi, -p3.hi);
      el = __fadd_rn(el, s1.lo);
      float rx = __fadd_rn(s1.hi, __fadd_rn(lo, el));
      lo = __fsub_rn(bi.lo, __fadd_rn(__fadd_rn(p4.lo, p5.lo), p6.lo));
      DF s2 = two_sum(bi.hi, -p4.hi);
      el = s2.lo;
      s2 = two_sum(s2.hi, -p5.hi);
      el = __fadd_rn(el, s2.lo);
      s2 = two_sum(s2.hi, -p6.hi);
      el = __fadd_rn(el, s2.lo);
      float ry = __fadd_rn(s2.hi, __fadd_rn(lo, el));
      rx *= scj;
      ry *= scj;
      if (bad) rx = ry = __int_as_float(0x7FC00000);
      rowr = __fmaf_rn(rx, rx, __fmaf_rn(ry, ry, rowr));
      o[(long long)(i0 + pr0 + q) * out.pitch + c] = make_float2(rx * oscale, ry * oscale);
    }
    ar = df_add(ar, DF{rowr, 0.f});
    buf ^= 1;
  }
  cp_async_wait_all();
  for (int off2 = 16; off2 > 0; off2 >>= 1) ar = df_add(ar, df_shfl_down(ar, off2));
  if (lane == 0) sh.redf[warp] = make_float2(ar.hi, ar.lo);
  __syncthreads();
  if (tid == 0) {
    DF s0 = {0.f, 0.f};
    for (int w = 0; w < kRxWarps; w++) s0 = df_add(s0, DF{sh.redf[w].x, sh.redf[w].y});
    part[(long long)j * gridDim.x + blockIdx.x] = (double)s0.hi + (double)s0.lo;
  }
}

}  // namespace

cudaError_t prepare_shift_residual_fx() {
  return cudaFuncSetAttribute(k_shift_residual_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSxSmem);
}

void launch_shift_residual_fx(cudaStream_t s, int gx, int N, int n, const double2 *z, const double2 *b,
                              const double2 *c1, double off, float oscale, const float *sc, View out,
                              const int *frozen, double *part) {
  dim3 grid(gx, n);
  k_shift_residual_fx<<<grid, kRxThreads, kSxSmem, s>>>(N, z, b, c1, off, oscale, sc, out, frozen, part);
}

}  // namespace pd
