// Residual of eq. (1) for the refinement without FP64 instructions (GB300 issues FP64 at
// 1/58 of its FP32 rate; measured 1.26 vs 73 TFLOP/s), for a bidiagonal time matrix:
//
//   r_k = fhat_k - bd_k u_k - bs_k u_{k+off} - (kappa/h^2)(4 u_k - sum of the 4 neighbours),
//   fhat_k = f_k + u0coef_k u0,
//
// output in FP32 (the refinement's next right-hand side) with its squared norm.
//
//   - Work item: one spatial tile (16 rows x 128 columns) and a run of consecutive time
//     steps, walked in the order in which u_{k+off} precedes u_k (ascending k for off = -1,
//     descending for off = +1).  The FP64 halo tile of the next step is copied into shared
//     memory by cp.async while the current one is computed, and each thread keeps its
//     points' u_k for the next step's bs term, so u is read once.
//   - Fixed point: the values of a halo tile are truncated to units of 2^-S, one scale per
//     tile and step, S = 1081 - (largest biased exponent in the tile), so every |value| <
//     2^59 units; the truncation, below 2^-58 max|u| of the tile, is under the FP64 rounding
//     of the largest value.  A value v is held as three FP32 limbs t2 2^42 + t1 2^21 + t0
//     (|t2| < 2^17, t1, t0 < 2^21, all of the value's sign), each an exact FP32 number.
//   - The stencil difference T1 = 4 u_k - (sum of neighbours), the cancellation-critical
//     part, is exact: per limb, 4 c - (sum of 4 neighbours) is an integer multiple of the
//     limb unit below 2^24 units, exact in FP32 arithmetic (FMA pipe, no integer work).
//   - The remaining arithmetic is float-float (pairs hi + lo of FP32) with the error-free
//     transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA product split:
//     every term is kept to about 2^-47 of its size and their hi parts are summed exactly,
//     so r is accurate to far below the FP64 rounding of the same formula (2^-53 of terms
//     of size 8 kappa/h^2 |u|).
//   - FP64 inputs become float-float by bit operations: hi = the value truncated to 24
//     significant bits, lo = the remaining 29 bits converted to FP32.
//   - Range: tiles whose largest |u| is below about 2^-88 (kappa/h^2 = 2^20) lose relative
//     accuracy in the u terms (the scaled constants become subnormal; below 2^-170 they
//     are 0); |u| >= 2^186, Inf or NaN in a tile makes that tile's r NaN.
#include <cstdint>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kRxRows = 16, kRxCols = 128, kRxThreads = 256;
constexpr int kRxHR = kRxRows + 2, kRxHC = kRxCols + 2;  // halo tile
constexpr int kRxHalo = kRxHR * kRxHC;
constexpr int kRxPer = (kRxHalo + kRxThreads - 1) / kRxThreads;  // halo values per thread
constexpr int kRxPts = kRxRows * kRxCols / kRxThreads;           // rows per thread (8)
constexpr int kRxWarps = kRxThreads / 32;

struct RxShared {
  unsigned long long raw[2][kRxHalo];  // FP64 bits of the halo tile, double-buffered
  float4 limb[kRxHalo];                // (t2 2^42, t1 2^21, t0, -) of each halo value
  unsigned red_e[kRxWarps];
  float2 cst[3];  // the step's bd_k, bs_k, u0coef_k as float-float pairs
  float2 redf[2][kRxWarps];
};
constexpr size_t kRxSmem = sizeof(RxShared);

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// exact when a = 0 or exponent(a) >= exponent(b)
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
// a * b as an unnormalised pair (p, e), p + e = a b to about 2^-47 |a b|
__device__ __forceinline__ DF df_mul_un(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return {p, __fadd_rn(__fmaf_rn(a.hi, b.hi, -p), __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi)))};
}

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

// 64-bit logical right shift; amounts of 64 and more give 0 (PTX shr clamps the amount)
__device__ __forceinline__ unsigned long long shr64(unsigned long long x, unsigned s) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}

// FP64 bits -> the three limbs of its fixed-point value in units 2^-S, S = 1081 - emax:
// v = m 2^(e - 1075 + S) = (m << 6) >> (emax - e) (m < 2^53, so m << 6 < 2^59; truncated
// below a unit), cut into 21-bit pieces and made FP32 by the mantissa trick at the limb's
// own exponent: the FP32 number X with t in the mantissa of 2^(23 + 21 j) is 2^(23 + 21 j)
// + t 2^(21 j), and X - 2^(23 + 21 j) is exact (here times the sign, in one FMA).  Zero and subnormal
// inputs (e = 0) are taken with the implicit bit: below 2^-1022 they only matter in a tile
// with emax < 64, where every scaled coefficient is 0.
__device__ __forceinline__ float4 to_limbs(unsigned long long bits, unsigned emax) {
  const uint32_t hw = (uint32_t)(bits >> 32), lw = (uint32_t)bits;
  const unsigned e = (hw >> 20) & 0x7FFu;
  const unsigned long long m = ((unsigned long long)((hw & 0xFFFFFu) | 0x100000u) << 32) | lw;
  const unsigned long long v = shr64(m << 6, emax - e);
  const uint32_t vl = (uint32_t)v, vh = (uint32_t)(v >> 32);
  const uint32_t t0 = vl & 0x1FFFFFu, t1 = __funnelshift_r(vl, vh, 21) & 0x1FFFFFu, t2 = vh >> 10;
  // sign: sg = +-1; sg (X - 2^(23 + 21 j)) as one exact FMA
  const float sg = __uint_as_float((hw & 0x80000000u) | 0x3F800000u);
  constexpr uint32_t E2 = 192u << 23, E1 = 171u << 23, E0 = 150u << 23;
  float4 l;
  l.x = __fmaf_rn(sg, __uint_as_float(E2 | t2), __fmul_rn(sg, -0x1p65f));
  l.y = __fmaf_rn(sg, __uint_as_float(E1 | t1), __fmul_rn(sg, -0x1p44f));
  l.z = __fmaf_rn(sg, __uint_as_float(E0 | t0), __fmul_rn(sg, -0x1p23f));
  l.w = 0.f;
  return l;
}

__device__ __forceinline__ DF df_shfl_down(DF a, int o) {
  return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Work items: item = chunk * tiles + tile; chunk q covers positions [q n / nch, (q+1) n / nch)
// of the walk order, position p being time step p (off = -1) or n - 1 - p (off = +1).
struct RxGeom {
  int N, n, off, tx, tiles, nch, items;
};
struct RxItem {
  int pbeg, pend, i0, c0;
};
__device__ __forceinline__ RxItem rx_item(const RxGeom &g, int it) {
  const int q = it / g.tiles, t = it - q * g.tiles;
  const int ty = t / g.tx;
  RxItem r;
  r.pbeg = (int)((long long)q * g.n / g.nch);
  r.pend = (int)((long long)(q + 1) * g.n / g.nch);
  r.i0 = ty * kRxRows;
  r.c0 = (t - ty * g.tx) * kRxCols;
  return r;
}
__device__ __forceinline__ int rx_step_k(const RxGeom &g, int p) { return g.off < 0 ? p : g.n - 1 - p; }

// the halo tile of u_k at (i0, c0) into raw: zero outside the grid.  Warp w copies halo
// rows w, w + 8, ...: per row one base address, the lanes' columns at fixed offsets.
__device__ __forceinline__ void issue_halo(unsigned long long *raw, const double *u, const RxGeom &g,
                                           int k, int i0, int c0) {
  const int N = g.N, lane = threadIdx.x & 31;
  const double *uk = u + (long long)k * N * N;
  const bool cols_in = c0 >= 1 && c0 + kRxCols < N;
  for (int hr = threadIdx.x >> 5; hr < kRxHR; hr += kRxWarps) {
    const int i = i0 - 1 + hr;
    unsigned long long *dst = raw + hr * kRxHC + lane;
    if ((unsigned)i >= (unsigned)N) {
#pragma unroll
      for (int j = 0; j < 4; j++) cp_async8(dst + 32 * j, u, 0);
      if (lane < kRxHC - 128) cp_async8(dst + 128, u, 0);
      continue;
    }
    const double *src = uk + (long long)i * N + (c0 - 1) + lane;
    if (cols_in) {
#pragma unroll
      for (int j = 0; j < 4; j++) cp_async8(dst + 32 * j, src + 32 * j, 8);
      if (lane < kRxHC - 128) cp_async8(dst + 128, src + 128, 8);
    } else {
#pragma unroll
      for (int j = 0; j < 5; j++) {
        const int hc = lane + 32 * j;
        if (j < 4 || hc < kRxHC) {
          const bool in = (unsigned)(c0 - 1 + hc) < (unsigned)N;
          cp_async8(dst + 32 * j, in ? src + 32 * j : u, in ? 8 : 0);
        }
      }
    }
  }
}

// FMODE 0: fhat from f and u0; 1: the same, and cached as float-float pairs in fc_out;
// 2: fhat read from the cache fc_in.  part[2 blockIdx.x] = sum |r|^2, part[2 blockIdx.x +
// 1] = sum |fhat|^2 when want_f.
template <int FMODE>
__global__ void __launch_bounds__(kRxThreads, 2)
k_residual_fx(RxGeom g, float *__restrict__ r, const double *__restrict__ u,
              const double *__restrict__ f, const double *__restrict__ u0,
              const double *__restrict__ u0coef, const double *__restrict__ bd,
              const double *__restrict__ bs, double ih2, int want_f, double *__restrict__ part,
              const float2 *__restrict__ fc_in, float2 *__restrict__ fc_out) {
  extern __shared__ __align__(16) unsigned char rx_smem[];
  RxShared &sh = *reinterpret_cast<RxShared *>(rx_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = g.N;
  const long long m = (long long)N * N;
  const int pc = tid % kRxCols, pr0 = (tid / kRxCols) * kRxPts;  // column, first row
  const DF ihd = split(ih2);  // kappa / h^2
  DF ar = {0.f, 0.f}, af = {0.f, 0.f};
  // this thread's u_{k+off}: the previous step's u_k in its units, or (at the first step of
  // an item) the FP64 bits read from memory
  float uph[kRxPts], upl[kRxPts];
#pragma unroll
  for (int t = 0; t < kRxPts; t++) uph[t] = upl[t] = 0.f;
  int s_prev = 0;
  bool bad_prev = false;

  int it = blockIdx.x;
  RxItem cur_it = {0, 0, 0, 0};
  int p = 0;
  // thread 0: bd_k, bs_k, u0coef_k of the coming step, read one step ahead
  double kbd = 0.0, kbs = 0.0, ku0 = 0.0;
  if (it < g.items) {
    cur_it = rx_item(g, it);
    p = cur_it.pbeg;
    const int k = rx_step_k(g, p);
    issue_halo(sh.raw[0], u, g, k, cur_it.i0, cur_it.c0);
    if (tid == 0) {
      kbd = bd[k];
      kbs = bs[k];
      if (FMODE != 2 && u0) ku0 = u0coef[k];
    }
  }
  cp_async_commit();
  int buf = 0;
  while (it < g.items) {
    cp_async_wait_all();
    __syncthreads();  // raw[buf] complete; the previous step is done with limb[] and red_*
    // the next step of this CTA: the next position of the item, or the next item
    int it2 = it, p2 = p + 1;
    RxItem nx = cur_it;
    if (p2 >= cur_it.pend) {
      it2 = it + gridDim.x;
      if (it2 < g.items) {
        nx = rx_item(g, it2);
        p2 = nx.pbeg;
      }
    }
    if (it2 < g.items) issue_halo(sh.raw[buf ^ 1], u, g, rx_step_k(g, p2), nx.i0, nx.c0);
    cp_async_commit();

    const int k = rx_step_k(g, p);
    const int kp = (k + g.off + g.n) % g.n;
    const bool have_prev = p > cur_it.pbeg;
    const int i0 = cur_it.i0, c0 = cur_it.c0, c = c0 + pc;
    // this step's fhat (or f) and, at the first step of an item, u_{k+off}: loads issued
    // now, used after the two barriers below
    // (rows t < nrow of the thread are inside the grid; x0 = offset of its first point)
    const int nrow = c < N ? min(kRxPts, N - i0 - pr0) : 0;
    const long long x0 = (long long)(i0 + pr0) * N + c;
    const long long kx0 = (long long)k * m + x0;  // the thread's first point in plane k
    float2 fq[kRxPts];
#pragma unroll
    for (int t = 0; t < kRxPts; t++) {
      const bool ok = t < nrow;
      if (FMODE == 2) {
        fq[t] = ok ? fc_in[kx0 + t * N] : make_float2(0.f, 0.f);
      } else {
        const double fv = ok ? f[kx0 + t * N] : 0.0;
        fq[t] = make_float2(__int_as_float(__double2hiint(fv)), __int_as_float(__double2loint(fv)));
      }
    }
    if (!have_prev) {
      const double *up0 = u + (long long)kp * m + x0;
#pragma unroll
      for (int t = 0; t < kRxPts; t++) {
        const double uv = t < nrow ? up0[t * N] : 0.0;
        uph[t] = __int_as_float(__double2hiint(uv));
        upl[t] = __int_as_float(__double2loint(uv));
      }
    }
    // per-step constants, split once per CTA; then those of the next step requested
    if (tid == 0) {
      const DF a = split(kbd), b = split(kbs), cc = split(ku0);
      sh.cst[0] = make_float2(a.hi, a.lo);
      sh.cst[1] = make_float2(b.hi, b.lo);
      sh.cst[2] = make_float2(cc.hi, cc.lo);
      if (it2 < g.items) {
        const int k2 = rx_step_k(g, p2);
        kbd = bd[k2];
        kbs = bs[k2];
        if (FMODE != 2 && u0) ku0 = u0coef[k2];
      }
    }
    // 1. largest exponent of the halo tile
    // (the largest high word without its sign bit has the largest exponent)
    const unsigned long long *raw = sh.raw[buf];
    unsigned emax = 0;
#pragma unroll
    for (int e = 0; e < kRxPer; e++) {
      const int q = tid + e * kRxThreads;
      if (q < kRxHalo) emax = max(emax, (unsigned)(raw[q] >> 32) & 0x7FFFFFFFu);
    }
    emax = __reduce_max_sync(0xffffffffu, emax) >> 20;
    if (lane == 0) sh.red_e[warp] = emax;
    __syncthreads();
    emax = 0;
#pragma unroll
    for (int w = 0; w < kRxWarps; w++) emax = max(emax, sh.red_e[w]);
    // 2. fixed-point limbs
#pragma unroll
    for (int e = 0; e < kRxPer; e++) {
      const int q = tid + e * kRxThreads;
      if (q < kRxHalo) sh.limb[q] = to_limbs(raw[q], emax);
    }
    __syncthreads();
    // (kappa/h^2) 2^-S and bd_k 2^-S multiply fixed-point values, and bs_k 2^-S' those of
    // the previous step (beyond S = 252, |u| < 2^-170: the products are 0)
    const bool bad = emax > 1081 + 126;  // Inf/NaN or |u| >= 2^186 in the tile
    const int S = 1081 - (int)emax;
    const int sc = S > 252 ? 252 : S;
    const DF c3 = df_scale_down(ihd, sc);
    const DF cb = df_scale_down(DF{sh.cst[0].x, sh.cst[0].y}, sc);
    const DF bsk = {sh.cst[1].x, sh.cst[1].y};
    const DF cs = have_prev ? df_scale_down(bsk, s_prev > 252 ? 252 : s_prev) : bsk;
    const bool nan_out = bad || (have_prev && bad_prev);
    const DF ck = {sh.cst[2].x, sh.cst[2].y};
    const bool has_u0 = FMODE != 2 && u0 && (ck.hi != 0.f || ck.lo != 0.f);

    // 3. the thread's points: column c0 + pc, rows i0 + pr0 .. + kRxPts - 1
    if (!have_prev) {
#pragma unroll
      for (int t = 0; t < kRxPts; t++) {
        const DF un = split_bits((uint32_t)__float_as_int(uph[t]), (uint32_t)__float_as_int(upl[t]));
        uph[t] = un.hi;
        upl[t] = un.lo;
      }
    }
    float rowr = 0.f, rowf = 0.f;
    const float4 *L = sh.limb + pc + 1;
    float4 up = L[pr0 * kRxHC], cu = L[(pr0 + 1) * kRxHC];
#pragma unroll
    for (int t = 0; t < kRxPts; t++) {
      const int hr = pr0 + t + 1;
      const float4 dn = L[(hr + 1) * kRxHC];
      const float4 lf = L[hr * kRxHC - 1], rt = L[hr * kRxHC + 1];
      const bool ok = t < nrow;
      // T1 per limb, exact; then as a float-float pair
      const float a2 = __fmaf_rn(4.f, cu.x, -__fadd_rn(__fadd_rn(up.x, dn.x), __fadd_rn(lf.x, rt.x)));
      const float a1 = __fmaf_rn(4.f, cu.y, -__fadd_rn(__fadd_rn(up.y, dn.y), __fadd_rn(lf.y, rt.y)));
      const float a0 = __fmaf_rn(4.f, cu.z, -__fadd_rn(__fadd_rn(up.z, dn.z), __fadd_rn(lf.z, rt.z)));
      DF t1 = two_sum(a2, a1);
      t1.lo = __fadd_rn(t1.lo, a0);
      DF uc = fast_two_sum(cu.x, cu.y);
      uc.lo = __fadd_rn(uc.lo, cu.z);
      const DF un = {uph[t], upl[t]};
      uph[t] = uc.hi;
      upl[t] = uc.lo;
      DF fh;
      if (FMODE == 2) {
        fh = {fq[t].x, fq[t].y};
      } else {
        fh = split_bits((uint32_t)__float_as_int(fq[t].x), (uint32_t)__float_as_int(fq[t].y));
        if (has_u0 && ok) fh = df_add(fh, df_mul(ck, split(u0[x0 + t * N])));
        if (FMODE == 1 && ok) fc_out[kx0 + t * N] = make_float2(fh.hi, fh.lo);
      }
      const DF p1 = df_mul_un(cb, uc), p2 = df_mul_un(cs, un), p3 = df_mul_un(c3, t1);
      // fhat - p1 - p2 - p3: the hi parts summed exactly, the low parts and errors in FP32
      const float lo = __fsub_rn(fh.lo, __fadd_rn(__fadd_rn(p1.lo, p2.lo), p3.lo));
      DF s = two_sum(fh.hi, -p1.hi);
      float el = s.lo;
      s = two_sum(s.hi, -p2.hi);
      el = __fadd_rn(el, s.lo);
      s = two_sum(s.hi, -p3.hi);
      el = __fadd_rn(el, s.lo);
      float rv = __fadd_rn(s.hi, __fadd_rn(lo, el));
      if (nan_out) rv = __int_as_float(0x7FC00000);
      if (ok) {
        r[kx0 + t * N] = rv;
        rowr = __fmaf_rn(rv, rv, rowr);
        if (want_f) {
          const float fv = __fadd_rn(fh.hi, fh.lo);
          rowf = __fmaf_rn(fv, fv, rowf);
        }
      }
      up = cu;
      cu = dn;
    }
    ar = df_add(ar, DF{rowr, 0.f});
    af = df_add(af, DF{rowf, 0.f});
    s_prev = S;
    bad_prev = bad;
    it = it2;
    cur_it = nx;
    p = p2;
    buf ^= 1;
  }
  cp_async_wait_all();
  // CTA sums: float-float over the warps, one conversion to FP64 per CTA
  for (int o = 16; o > 0; o >>= 1) {
    ar = df_add(ar, df_shfl_down(ar, o));
    af = df_add(af, df_shfl_down(af, o));
  }
  if (lane == 0) {
    sh.redf[0][warp] = make_float2(ar.hi, ar.lo);
    sh.redf[1][warp] = make_float2(af.hi, af.lo);
  }
  __syncthreads();
  if (tid == 0) {
    DF s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
    for (int w = 0; w < kRxWarps; w++) {
      s0 = df_add(s0, DF{sh.redf[0][w].x, sh.redf[0][w].y});
      s1 = df_add(s1, DF{sh.redf[1][w].x, sh.redf[1][w].y});
    }
    part[2 * blockIdx.x] = (double)s0.hi + (double)s0.lo;
    part[2 * blockIdx.x + 1] = (double)s1.hi + (double)s1.lo;
  }
}

template <int FMODE>
void launch_mode(cudaStream_t s, int blocks, const RxGeom &g, float *r, const double *u,
                 const double *f, const double *u0, const double *u0coef, const double *bd,
                 const double *bs, double ih2, bool want_f, double *part, const float2 *fc_in,
                 float2 *fc_out) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_residual_fx<FMODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kRxSmem);
    attr = true;
  }
  k_residual_fx<FMODE><<<blocks, kRxThreads, kRxSmem, s>>>(g, r, u, f, u0, u0coef, bd, bs, ih2,
                                                           want_f ? 1 : 0, part, fc_in, fc_out);
}


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
                    const double2 *__restrict__ c1, double off, float oscale, View out,
                    const int *__restrict__ frozen, double *__restrict__ part) {
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

int residual_fx_blocks(int num_sms) { return 2 * num_sms; }

void launch_residual_fx(cudaStream_t s, int blocks, int N, int n, int off, double kappa, float *r,
                        const double *u, const double *f, const double *u0, const double *u0coef,
                        const double *bd, const double *bs, bool want_f, double *part,
                        const float2 *fc_in, float2 *fc_out) {
  const double h = 1.0 / (N + 1);
  RxGeom g;
  g.N = N;
  g.n = n;
  g.off = off < 0 ? -1 : 1;
  g.tx = (N + kRxCols - 1) / kRxCols;
  g.tiles = g.tx * ((N + kRxRows - 1) / kRxRows);
  // time-step runs: enough items for about eight per CTA (the tail of a static
  // distribution then costs little), runs of at least two steps
  g.nch = 1;
  while ((long long)g.tiles * g.nch < 8ll * blocks && n / (2 * g.nch) >= 2) g.nch *= 2;
  g.items = g.tiles * g.nch;
  const double ih2 = kappa / (h * h);
  if (fc_in)
    launch_mode<2>(s, blocks, g, r, u, f, u0, u0coef, bd, bs, ih2, want_f, part, fc_in, nullptr);
  else if (fc_out)
    launch_mode<1>(s, blocks, g, r, u, f, u0, u0coef, bd, bs, ih2, want_f, part, nullptr, fc_out);
  else
    launch_mode<0>(s, blocks, g, r, u, f, u0, u0coef, bd, bs, ih2, want_f, part, nullptr, nullptr);
}


void launch_shift_residual_fx(cudaStream_t s, int N, int n, const double2 *z, const double2 *b,
                              const double2 *c1, double off, float oscale, View out,
                              const int *frozen, double *part) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_shift_residual_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSxSmem);
    attr = true;
  }
  dim3 grid(shift_residual_blocks(N, n), n);
  k_shift_residual_fx<<<grid, kRxThreads, kSxSmem, s>>>(N, z, b, c1, off, oscale, out, frozen, part);
}

}  // namespace pd
