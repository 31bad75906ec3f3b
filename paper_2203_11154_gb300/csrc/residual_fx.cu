// Residual of eq. (1) for the refinement without FP64 instructions (GB300 issues FP64 at
// 1/58 of its FP32 rate; measured 1.26 vs 73 TFLOP/s), for a bidiagonal time matrix:
//
//   r_k = fhat_k - bd_k u_k - bs_k u_{k+off} - (kappa/h^2)(4 u_k - sum of the 4 neighbours),
//   fhat_k = f_k + u0coef_k u0,
//
// output in FP32 (the refinement's next right-hand side) with its squared norm.
//
//   - The stencil difference T1 = 4 u_k - (sum of neighbours) is the cancellation-critical
//     part: it is computed exactly in 64-bit integers.  The FP64 values of a tile (16 rows x
//     128 columns of one u_k plus the halo) are converted, by bit operations, to fixed point
//     with one scale per tile, 2^-S with S = 1081 - (largest biased exponent in the tile), so
//     every |value| < 2^59 units and |T1| < 2^62; the conversion truncates below one unit,
//     2^-S <= 2^-58 max|u|, an error below the FP64 rounding of the largest value.
//   - The remaining terms are formed in float-float (pairs hi + lo of FP32) with the
//     error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA
//     product split, about 2^-46 relative per term: r is accurate to far below the FP64
//     rounding of the same formula (2^-53 of terms of size 8 kappa/h^2 |u|).
//   - FP64 inputs become float-float by bit operations: hi = the value truncated to 24
//     significant bits, lo = the remaining 29 bits converted to FP32.
#include <cstdint>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kFxRows = 32, kFxCols = 128, kFxThreads = 256;
constexpr int kFxHR = kFxRows + 2, kFxHC = kFxCols + 2;  // halo tile

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }

// 2^e as FP32 for e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// x * 2^-s for s in [-126, 252] (two exact power-of-two products; flushes below 2^-149)
__device__ __forceinline__ float scale_down(float x, int s) {
  const int a = s >> 1;
  return __fmul_rn(__fmul_rn(x, pow2f(-a)), pow2f(a - s));
}
__device__ __forceinline__ DF df_scale_down(DF x, int s) { return {scale_down(x.hi, s), scale_down(x.lo, s)}; }

// Integer -> FP32 without a conversion instruction (conversions issue on GB300's slow
// FP64 pipe): for 0 <= x < 2^23, the FP32 number with x in the mantissa of 2^23 is
// 2^23 + x exactly; subtracting 2^23 leaves x.
__device__ __forceinline__ float u23_to_float(unsigned x) {
  return __fsub_rn(__uint_as_float(0x4B000000u | x), 8388608.f);
}

// FP64 bits -> float-float: |x| >= 2^-100 kept (hi truncated to 24 bits, lo the rest,
// rounded to 24 bits), smaller values are 0; Inf/NaN give NaN
__device__ __forceinline__ DF split_bits(uint32_t hw, uint32_t lw) {
  const int e = (int)((hw >> 20) & 0x7FFu);
  if (e == 0x7FF || e > 1023 + 127) return {__int_as_float(0x7FC00000), 0.f};
  if (e < 1023 - 100) return {0.f, 0.f};
  const uint32_t sign = hw & 0x80000000u;
  const float hi = __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  // remaining 29 bits, weight 2^(e - 1075), e - 1075 in [-152, 52]
  const int ex = e - 1075;
  const int a = ex >> 1;
  const unsigned rem = lw & 0x1FFFFFFFu;  // 29 bits = 23 high + 6 low
  const float remf = __fmaf_rn(u23_to_float(rem >> 6), 64.f, u23_to_float(rem & 63u));
  float lo = __fmul_rn(__fmul_rn(remf, pow2f(a)), pow2f(ex - a));
  if (sign) lo = -lo;
  return {hi, lo};
}

__device__ __forceinline__ DF split(double x) {
  return split_bits((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x));
}

// FP64 bits -> fixed point with 2^-S units (S = 1081 - e_max from the tile's largest
// biased exponent e_max, see above): m 2^(e-1075) 2^S = (m << 6) >> (e_max - e), one
// branch-free right shift (m < 2^53, so m << 6 < 2^59 loses nothing); truncated below a unit
__device__ __forceinline__ long long to_fixed(uint32_t hw, uint32_t lw, int S) {
  const int e = (int)((hw >> 20) & 0x7FFu);
  const unsigned long long m = ((unsigned long long)((hw & 0xFFFFFu) | 0x100000u) << 32) | lw;
  const int rs = 1081 - S - e;  // >= 0
  const unsigned long long v = (e == 0 || rs >= 64) ? 0ull : ((m << 6) >> rs);
  const long long sv = (long long)v;
  return (hw & 0x80000000u) ? -sv : sv;
}

// 64-bit integer |v| < 2^62 -> float-float, about 2^-47 relative.  64-bit integer <-> float
// conversions run on the FP64 pipe, so v is cut into three 21-bit chunks that FP32 holds
// exactly, v = t2 2^42 + t1 2^21 + t0 (t2 signed), and summed error-free.
__device__ __forceinline__ DF df_from_ll(long long v) {
  const unsigned lo32 = (unsigned)v, hi32 = (unsigned)((unsigned long long)v >> 32);
  const int t2 = (int)hi32 >> 10;
  const unsigned t1 = __funnelshift_r(lo32, hi32, 21) & 0x1FFFFFu;
  const unsigned t0 = lo32 & 0x1FFFFFu;
  // t2 in [-2^20, 2^20): offset by 2^20 into [0, 2^21)
  const float f2 = __fsub_rn(u23_to_float((unsigned)(t2 + (1 << 20))), 1048576.f);
  DF s = two_sum(__fmul_rn(f2, 4398046511104.f),                 // 2^42
                 __fmul_rn(u23_to_float(t1), 2097152.f));         // 2^21
  s.lo = __fadd_rn(s.lo, u23_to_float(t0));
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DF df_shfl_down(DF a, int o) {
  return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

// grid-stride over tiles (x tile, y tile, k); part[2 * blockIdx.x] = sum |r|^2 (FP32 per
// tile), part[2 * blockIdx.x + 1] = sum |fhat|^2 when want_f
__global__ void __launch_bounds__(kFxThreads, 4)
k_residual_fx(int N, int n, int off, float *__restrict__ r, const double *__restrict__ u,
              const double *__restrict__ f, const double *__restrict__ u0,
              const double *__restrict__ u0coef, const double *__restrict__ bd,
              const double *__restrict__ bs, double ih2, int want_f, double *__restrict__ part,
              const float2 *__restrict__ fc_in, float2 *__restrict__ fc_out) {
  __shared__ long long sfx[kFxHR * kFxHC];
  __shared__ unsigned red_e[kFxThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long m = (long long)N * N;
  const int tx = (N + kFxCols - 1) / kFxCols, ty = (N + kFxRows - 1) / kFxRows;
  const long long tiles = (long long)tx * ty * n;
  const DF ihd = split(ih2);  // kappa / h^2
  // per-thread sums of the per-tile FP32 sums in float-float (no FP64 arithmetic)
  DF ar = {0.f, 0.f}, af = {0.f, 0.f};
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int k = (int)(t / ((long long)tx * ty));
    const int rem = (int)(t - (long long)k * tx * ty);
    const int i0 = (rem / tx) * kFxRows, c0 = (rem % tx) * kFxCols;
    const int kp = (k + off + n) % n;
    const double *uk = u + (long long)k * m;
    // 1. halo tile of u_k: raw bits into shared memory, largest exponent
    unsigned emax = 0;
    for (int q = tid; q < kFxHR * kFxHC; q += kFxThreads) {
      const int hr = q / kFxHC, hc = q - hr * kFxHC;
      const int i = i0 - 1 + hr, c = c0 - 1 + hc;
      long long bits = 0;
      if (i >= 0 && i < N && c >= 0 && c < N) bits = __double_as_longlong(uk[(long long)i * N + c]);
      sfx[q] = bits;
      emax = max(emax, (unsigned)((bits >> 52) & 0x7FF));
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (lane == 0) red_e[warp] = emax;
    __syncthreads();
    emax = 0;
#pragma unroll
    for (int w = 0; w < kFxThreads / 32; w++) emax = max(emax, red_e[w]);
    // Inf/NaN, or |u| >= 2^186 (beyond the scaling range below): the tile's residual is NaN
    const bool bad = emax > 1081 + 126;
    const int S = 1081 - (int)emax;
    // 2. to fixed point in place
    for (int q = tid; q < kFxHR * kFxHC; q += kFxThreads) {
      const long long bits = sfx[q];
      sfx[q] = to_fixed((uint32_t)(bits >> 32), (uint32_t)bits, S);
    }
    __syncthreads();
    // per-tile constants, float-float: (kappa/h^2) 2^-S and bd_k 2^-S multiply fixed-point
    // values (beyond S = 252, |u| < 2^-170: those products flush to 0)
    const int sc = S > 252 ? 252 : S;
    const DF c3 = df_scale_down(ihd, sc);
    const DF cb = df_scale_down(split(bd[k]), sc);
    const DF bsk = split(bs[k]);
    const DF ck = u0 ? split(u0coef[k]) : DF{0.f, 0.f};
    const bool has_u0 = ck.hi != 0.f || ck.lo != 0.f;
    // 3. the tile's points: thread -> column c0 + (tid % 128), rows (tid / 128) + 2 q
    const int pc = tid % kFxCols, pr0 = tid / kFxCols;
    const int c = c0 + pc;
    float rowr = 0.f, rowf = 0.f;
    if (c < N) {
#pragma unroll 4
      for (int pr = pr0; pr < kFxRows; pr += kFxThreads / kFxCols) {
        const int i = i0 + pr;
        if (i >= N) break;
        const int q = (pr + 1) * kFxHC + (pc + 1);
        const long long uc = sfx[q];
        const long long t1 = 4 * uc - (sfx[q - 1] + sfx[q + 1] + sfx[q - kFxHC] + sfx[q + kFxHC]);
        const long long x = (long long)i * N + c;
        // fhat in float-float: from the cache of an earlier residual of the same solve, or
        // from f and u0 (and then cached when asked)
        DF acc;
        if (fc_in) {
          const float2 q = fc_in[(long long)k * m + x];
          acc = {q.x, q.y};
        } else {
          acc = split(f[(long long)k * m + x]);
          if (has_u0) acc = df_add(acc, df_mul(ck, split(u0[x])));
          if (fc_out) fc_out[(long long)k * m + x] = make_float2(acc.hi, acc.lo);
        }
        DF fh = acc;
        acc = df_add(acc, df_neg(df_mul(cb, df_from_ll(uc))));
        acc = df_add(acc, df_neg(df_mul(bsk, split(u[(long long)kp * m + x]))));
        acc = df_add(acc, df_neg(df_mul(c3, df_from_ll(t1))));
        float rv = __fadd_rn(acc.hi, acc.lo);
        if (bad) rv = __int_as_float(0x7FC00000);
        r[(long long)k * m + x] = rv;
        rowr = __fmaf_rn(rv, rv, rowr);
        if (want_f) {
          const float fv = __fadd_rn(fh.hi, fh.lo);
          rowf = __fmaf_rn(fv, fv, rowf);
        }
      }
    }
    ar = df_add(ar, DF{rowr, 0.f});
    af = df_add(af, DF{rowf, 0.f});
    __syncthreads();  // the shared tile is reused by the next tile
  }
  // CTA sums: float-float over the warps, one conversion to FP64 per CTA
  for (int o = 16; o > 0; o >>= 1) {
    ar = df_add(ar, df_shfl_down(ar, o));
    af = df_add(af, df_shfl_down(af, o));
  }
  __shared__ DF redf[2][kFxThreads / 32];
  if (lane == 0) {
    redf[0][warp] = ar;
    redf[1][warp] = af;
  }
  __syncthreads();
  if (tid == 0) {
    DF s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
    for (int w = 0; w < kFxThreads / 32; w++) {
      s0 = df_add(s0, redf[0][w]);
      s1 = df_add(s1, redf[1][w]);
    }
    part[2 * blockIdx.x] = (double)s0.hi + (double)s0.lo;
    part[2 * blockIdx.x + 1] = (double)s1.hi + (double)s1.lo;
  }
}

}  // namespace

int residual_fx_blocks(int num_sms) { return 8 * num_sms; }

void launch_residual_fx(cudaStream_t s, int blocks, int N, int n, int off, double kappa, float *r,
                        const double *u, const double *f, const double *u0, const double *u0coef,
                        const double *bd, const double *bs, bool want_f, double *part,
                        const float2 *fc_in, float2 *fc_out) {
  const double h = 1.0 / (N + 1);
  k_residual_fx<<<blocks, kFxThreads, 0, s>>>(N, n, off, r, u, f, u0, u0coef, bd, bs,
                                              kappa / (h * h), want_f ? 1 : 0, part, fc_in, fc_out);
}

}  // namespace pd
