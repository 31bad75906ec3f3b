// Residual of eq. (1) for the refinement without FP64 instructions (GB300 issues FP64 at
// 1/58 of its FP32 rate), for a bidiagonal time matrix, as warp streams:
//
//   r_k = fhat_k - bd_k u_k - bs_k u_{k+off} - (kappa/h^2)(4 u_k - sum of the 4 neighbours),
//   fhat_k = f_k + u0coef_k u0,
//
// output in FP32 times a power of two `oscale` (the refinement keeps its FP32 right-hand
// sides near unit size whatever the scale of the data), with the sums of |oscale r|^2 and
// of |fscale fhat|^2.
//
//   - Work item of a warp: a strip of 30 output columns (lanes 1..30; lanes 0 and 31 carry
//     the halo columns) by kWsR = 6 rows, walked through a run of consecutive time steps in
//     the order in which u_{k+off} precedes u_k (ascending k for off = -1, descending for
//     off = +1).  A lane holds its column's kWsR + 2 values of u_k in registers: vertical
//     neighbours are its own, horizontal ones come from the adjacent lanes by shuffles.
//     The next step's column is loaded while the current one is computed, and a lane keeps
//     its points' u_k for the next step's bs term, so u is read from memory once (plus the
//     halo rows and columns, from L2).  No shared memory and no barrier until the final
//     CTA sum.
//   - Packed arithmetic: output rows t and t + 3 of a tile are the two components of every
//     FP32 operation (FADD2 / FMUL2 / FFMA2), each component rounded exactly as the scalar
//     operation, so the results are those of the scalar formulas bit for bit.
//   - Interior and edge tiles are two kernels: the interior one (every row and column the
//     tile reads inside the grid) loads without bounds checks; the edge one takes the
//     remaining tiles (enumerated directly) in short runs of time steps.  Compiled apart,
//     each keeps its state in registers (compiled together they spilled).
//   - Fixed point: one scale per warp tile and step, 2^-S with S = 1081 - (largest biased
//     exponent of the tile's (kWsR + 2) x 32 values, a warp max); every value becomes three
//     exact FP32 limbs (ff::limb_bits, ff::limbs2), so the stencil difference 4 u_k - (sum of the
//     neighbours), where the cancellation happens, is exact in FP32 arithmetic.
//   - The other terms are float-float pairs: fhat (split from FP64 by bit operations, or
//     read back from the float-float cache the first residual of a solve writes), the three
//     products with constants split on the host; their hi parts are summed with TwoSum and
//     the low parts and rounding errors in FP32, so r carries an error near 2^-47 of the
//     terms' size, far below the FP64 rounding of the same formula.
//   - Range: a tile whose largest |u| is 2^186 or more, Inf or NaN gives NaN residuals;
//     below about 2^-88 (kappa/h^2 = 2^20) the u terms lose relative accuracy.
#include <cstdint>

#include "ff.cuh"
#include "pd_internal.h"

#include <algorithm>

namespace pd {
namespace {

using namespace ff;

constexpr int kWsR = 6;      // output rows of a warp tile
constexpr int kWsOut = 30;   // output columns of a warp strip
constexpr int kWsWarps = 8;  // warps per CTA
constexpr int kWsThreads = 32 * kWsWarps;

// Tile sets of the warp-tile kernels (tiles of R rows by kWsOut output columns, strip sx
// starting at column c0 = kWsOut sx - 1): a tile is interior when its rows i0 - 1 .. i0 + R
// and the strip's 32 columns c0 .. c0 + 31 all lie inside the grid, i.e. row blocks
// [1, ty_in] and strips [1, tx_in].  The edge set is the row blocks outside [1, ty_in] (all
// strips), then strip 0 and the strips beyond tx_in of the row blocks inside.
struct TileGeom {
  int tx, ty, tx_in, ty_in;
};
__host__ __device__ __forceinline__ TileGeom tile_geom(int N, int R) {
  TileGeom g;
  g.tx = (N + kWsOut - 1) / kWsOut;
  g.ty = (N + R - 1) / R;
  g.tx_in = N > 31 ? (N - 31) / kWsOut : 0;
  g.ty_in = N > 1 + R ? (N - 1) / R - 1 : 0;
  if (g.tx_in == 0 || g.ty_in == 0) g.tx_in = g.ty_in = 0;
  return g;
}
__host__ __device__ __forceinline__ int tile_count(const TileGeom &g, bool interior) {
  const int in = g.tx_in * g.ty_in;
  return interior ? in : g.tx * g.ty - in;
}
// tile t of the interior or the edge set -> (row block, strip)
__device__ __forceinline__ void tile_at(const TileGeom &g, bool interior, int t, int &by, int &sx) {
  if (interior) {
    by = 1 + t / g.tx_in;
    sx = 1 + t % g.tx_in;
    return;
  }
  const int e1 = (g.ty - g.ty_in) * g.tx;
  if (t < e1) {
    const int fr = t / g.tx;
    sx = t - fr * g.tx;
    by = fr == 0 ? 0 : g.ty_in + fr;
  } else {
    const int ns = g.tx - g.tx_in, e2 = t - e1;
    by = 1 + e2 / ns;
    const int k = e2 - (by - 1) * ns;
    sx = k == 0 ? 0 : g.tx_in + k;
  }
}

// item = chunk * tiles + tile (tiles: the kernel's tile set); chunk q covers the positions
// [q n / nch, (q + 1) n / nch) of the time walk, position p being step p (off = -1) or
// n - 1 - p (off = +1)
struct WsGeom {
  int N, n, off, tiles, nch, items;
  TileGeom tg;
};

__device__ __forceinline__ int ws_step(const WsGeom &g, int p) { return g.off < 0 ? p : g.n - 1 - p; }

// FMODE 0: fhat from f and u0; 1: the same, also written to the cache fc_out as float-float
// pairs; 2: fhat read from the cache fc_in.  kbd[k] = (bd_k, bs_k) and ku0[k] = u0coef_k as
// float-float pairs, ihd = kappa / h^2 likewise.  part[2 b] = sum |oscale r|^2,
// part[2 b + 1] = sum |fscale fhat|^2 (when want_f) of CTA b.
struct WsArgs {
  float *r;
  const double *u, *f, *u0;
  const float4 *kbd;
  const float2 *ku0;
  DF ihd;
  float oscale, fscale;
  int want_f;
  const float2 *fc_in;
  float2 *fc_out;
};

// horizontal neighbours of both components from the adjacent lanes, summed
__device__ __forceinline__ float2 shfl_sum2(float2 v) {
  return add2(make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1)),
              make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1)));
}
// 4 c - (u + d + the horizontal neighbours of c) of one limb, exact
__device__ __forceinline__ float2 stencil2(float2 u, float2 c, float2 d) {
  return fma2(bc2(4.f), c, neg2(add2(add2(u, d), shfl_sum2(c))));
}

// One work item: the tile at rows i0.., the lane's column c, time-walk chunk q.  Output rows
// t and t + 3 (t < 3) are the components of the packed operations; Q[e] holds the limbs of
// rows e and e + 3 of the column (rows i0 - 1 + e), so output pair t reads Q[t] (above),
// Q[t + 1] (centre) and Q[t + 2] (below).
template <int FMODE, bool FULL>
__device__ __forceinline__ void ws_item(const WsGeom &g, const WsArgs &A, int q, int i0, int c,
                                        int lane, DF &ar, DF &af) {
  constexpr int R = kWsR;
  constexpr int H = R / 2;
  static_assert(R == 6, "packed row pairs (t, t + 3)");
  const int N = g.N;
  const long long m = (long long)N * N;
  const int pbeg = (int)((long long)q * g.n / g.nch), pend = (int)((long long)(q + 1) * g.n / g.nch);
  const bool cin = FULL || (unsigned)c < (unsigned)N;
  const bool outc = lane >= 1 && lane <= kWsOut && cin;
  const int nr = FULL ? R : min(R, N - i0);  // output rows inside the grid
  const long long cc = cin ? c : 0;
  // the scaling of output rows (t, t + 3): oscale, 0 outside the grid (so that they add
  // nothing to the sums)
  float2 osc[H];
#pragma unroll
  for (int t = 0; t < H; t++)
    osc[t] = make_float2(outc && t < nr ? A.oscale : 0.f, outc && t + H < nr ? A.oscale : 0.f);
  const long long rb = (long long)(i0 - 1) * N + cc;  // row i0 - 1 of the lane's column
  // the lane's column of one time step, rows i0 - 1 .. i0 + R (zero outside the grid)
  unsigned long long raw[R + 2];
  auto load_u = [&](int k) {
    const double *uk = A.u + (long long)k * m + rb;
#pragma unroll
    for (int e = 0; e < R + 2; e++) {
      const bool ok = FULL || (cin && (unsigned)(i0 - 1 + e) < (unsigned)N);
      raw[e] = ok ? (unsigned long long)__double_as_longlong(uk[(long long)e * N]) : 0ull;
    }
  };
  load_u(ws_step(g, pbeg));
  DF2 un[H];  // u_{k+off} of rows (t, t + 3), in the previous step's units
  int s_prev = 0;
  bool bad_prev = false;
  for (int p = pbeg; p < pend; p++) {
    const int k = ws_step(g, p);
    const bool first = p == pbeg;
    const long long kx0 = (long long)k * m + rb + N;  // the lane's row i0 in plane k
    // this step's fhat (cache) or f of the lane's points: 64-bit words
    unsigned long long fb[R];
#pragma unroll
    for (int t = 0; t < R; t++) {
      const bool ok = FULL || (outc && t < nr);
      if (FMODE == 2)
        fb[t] = ok ? *reinterpret_cast<const unsigned long long *>(A.fc_in + kx0 + (long long)t * N) : 0ull;
      else
        fb[t] = ok ? (unsigned long long)__double_as_longlong(A.f[kx0 + (long long)t * N]) : 0ull;
    }
    // first step of the item: u_{k+off} from memory (FP64, split below)
    unsigned long long ub[R];
    if (first) {
      const int kp = (k + g.off + g.n) % g.n;
      const double *up = A.u + (long long)kp * m + rb + N;
#pragma unroll
      for (int t = 0; t < R; t++)
        ub[t] = (outc && t < nr) ? (unsigned long long)__double_as_longlong(up[(long long)t * N]) : 0ull;
    }
    // largest exponent of the warp tile (the largest high word without its sign bit has
    // the largest exponent), then the limbs
    unsigned em = 0;
#pragma unroll
    for (int e = 0; e < R + 2; e++) em = max(em, (unsigned)(raw[e] >> 32) & 0x7FFFFFFFu);
    em = __reduce_max_sync(0xffffffffu, em) >> 20;
    LimbBits lb[R + 2];
#pragma unroll
    for (int e = 0; e < R + 2; e++) lb[e] = limb_bits(raw[e], em);
    Limbs2 Q[H + 2];
#pragma unroll
    for (int e = 0; e < H + 2; e++) Q[e] = limbs2(lb[e], lb[e + H]);
    // the next step's column, while this one is computed
    if (p + 1 < pend) load_u(ws_step(g, p + 1));
    const float4 kb = A.kbd[k];
    // (kappa/h^2) 2^-S and bd_k 2^-S multiply fixed-point values, bs_k 2^-S' those of the
    // previous step (beyond S = 252, |u| < 2^-170: the products are 0)
    const bool bad = em > 1081 + 126;  // Inf/NaN or |u| >= 2^186 in the tile
    const int S = 1081 - (int)em, sc = S > 252 ? 252 : S;
    const DF c3 = df_scale_down(A.ihd, sc);
    const DF cb = df_scale_down(DF{kb.x, kb.y}, sc);
    const DF cs = first ? DF{kb.z, kb.w} : df_scale_down(DF{kb.z, kb.w}, s_prev > 252 ? 252 : s_prev);
    const DF2 c32 = {bc2(c3.hi), bc2(c3.lo)}, cb2 = {bc2(cb.hi), bc2(cb.lo)}, cs2 = {bc2(cs.hi), bc2(cs.lo)};
    const bool nan_out = bad || (!first && bad_prev);
    DF ck = {0.f, 0.f};
    bool has_u0 = false;
    if (FMODE != 2 && A.u0) {
      const float2 c2 = A.ku0[k];
      ck = DF{c2.x, c2.y};
      has_u0 = c2.x != 0.f || c2.y != 0.f;
    }
    if (first) {
#pragma unroll
      for (int t = 0; t < H; t++) {
        const DF a = split_bits((uint32_t)(ub[t] >> 32), (uint32_t)ub[t]);
        const DF b = split_bits((uint32_t)(ub[t + H] >> 32), (uint32_t)ub[t + H]);
        un[t] = DF2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
      }
    }
    float2 rowr = make_float2(0.f, 0.f);
    float rowf = 0.f;
#pragma unroll
    for (int t = 0; t < H; t++) {
      // the exact stencil difference per limb, then as a float-float pair
      const Limbs2 &U = Q[t], &C = Q[t + 1], &D = Q[t + 2];
      const float2 a2 = stencil2(U.l2, C.l2, D.l2);
      const float2 a1 = stencil2(U.l1, C.l1, D.l1);
      const float2 a0 = stencil2(U.l0, C.l0, D.l0);
      DF2 t1 = two_sum2(a2, a1);
      t1.lo = add2(t1.lo, a0);
      DF2 uc = fast_two_sum2(C.l2, C.l1);
      uc.lo = add2(uc.lo, C.l0);
      const DF2 unt = un[t];
      un[t] = uc;
      // fhat of rows t and t + 3
      DF fa, fz;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int tt = t + h * H;
        const bool ok = outc && tt < nr;
        DF fh;
        if (FMODE == 2) {
          fh = DF{__uint_as_float((uint32_t)fb[tt]), __uint_as_float((uint32_t)(fb[tt] >> 32))};
        } else {
          fh = split_bits((uint32_t)(fb[tt] >> 32), (uint32_t)fb[tt]);
          if (has_u0 && ok) fh = df_add(fh, df_mul(ck, split(A.u0[rb + (long long)(tt + 1) * N])));
          if (FMODE == 1 && ok) A.fc_out[kx0 + (long long)tt * N] = make_float2(fh.hi, fh.lo);
          if (A.want_f && ok) {
            const float fv = __fmul_rn(__fadd_rn(fh.hi, fh.lo), A.fscale);
            rowf = __fmaf_rn(fv, fv, rowf);
          }
        }
        if (h == 0) fa = fh;
        else fz = fh;
      }
      const DF2 fh = {make_float2(fa.hi, fz.hi), make_float2(fa.lo, fz.lo)};
      const DF2 p1 = mul_un2(cb2, uc), p2 = mul_un2(cs2, unt), p3 = mul_un2(c32, t1);
      // fhat - p1 - p2 - p3: the hi parts summed exactly, the low parts and errors in FP32
      const float2 lo = sub2(fh.lo, add2(add2(p1.lo, p2.lo), p3.lo));
      DF2 s = two_sum2(fh.hi, neg2(p1.hi));
      float2 el = s.lo;
      s = two_sum2(s.hi, neg2(p2.hi));
      el = add2(el, s.lo);
      s = two_sum2(s.hi, neg2(p3.hi));
      el = add2(el, s.lo);
      float2 o = osc[t];
      if (nan_out) o = bc2(__int_as_float(0x7FC00000));
      const float2 rv = mul2(add2(s.hi, add2(lo, el)), o);
      if (outc && t < nr) A.r[kx0 + (long long)t * N] = rv.x;
      if (outc && t + H < nr) A.r[kx0 + (long long)(t + H) * N] = rv.y;
      rowr = fma2(rv, rv, rowr);
    }
    ar = df_add(ar, DF{__fadd_rn(rowr.x, rowr.y), 0.f});
    if (A.want_f) af = df_add(af, DF{rowf, 0.f});
    s_prev = S;
    bad_prev = bad;
  }
}

// FULL: the interior tiles, else the edge tiles.  CTA sums: float-float over the warps, one
// conversion to FP64 per CTA.
template <int FMODE, bool FULL>
__global__ void __launch_bounds__(kWsThreads, 2)
k_residual_ws(const __grid_constant__ WsGeom g, const __grid_constant__ WsArgs A,
              double *__restrict__ part) {
  constexpr int R = kWsR;
  __shared__ float2 red[2][kWsWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  DF ar = {0.f, 0.f}, af = {0.f, 0.f};
  for (int it = blockIdx.x * kWsWarps + warp; it < g.items; it += gridDim.x * kWsWarps) {
    const int q = it / g.tiles, t0 = it - q * g.tiles;
    int by, sx;
    tile_at(g.tg, FULL, t0, by, sx);
    ws_item<FMODE, FULL>(g, A, q, by * R, sx * kWsOut - 1 + lane, lane, ar, af);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar = df_add(ar, df_shfl_down(ar, o));
    af = df_add(af, df_shfl_down(af, o));
  }
  if (lane == 0) {
    red[0][warp] = make_float2(ar.hi, ar.lo);
    red[1][warp] = make_float2(af.hi, af.lo);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    DF s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
    for (int w = 0; w < kWsWarps; w++) {
      s0 = df_add(s0, DF{red[0][w].x, red[0][w].y});
      s1 = df_add(s1, DF{red[1][w].x, red[1][w].y});
    }
    part[2 * blockIdx.x] = (double)s0.hi + (double)s0.lo;
    part[2 * blockIdx.x + 1] = (double)s1.hi + (double)s1.lo;
  }
}

// time-step runs: enough items for about eight per warp (the tail of a static
// distribution then costs little), runs of at least two steps
void ws_chunks(WsGeom &g, int blocks) {
  const long long warps = (long long)blocks * kWsWarps;
  g.nch = 1;
  while ((long long)g.tiles * g.nch < 8 * warps && g.n / (2 * g.nch) >= 2) g.nch *= 2;
  g.items = g.tiles * g.nch;
}

// the interior kernel on `blocks` CTAs (partial sums part[0 .. 2 blocks)), then the edge
// kernel on `blocks_edge` CTAs (part[2 blocks ..))
template <int FMODE>
void launch_ws(cudaStream_t s, int blocks, int blocks_edge, int N, int n, int off, const WsArgs &A,
               double *part) {
  WsGeom g;
  g.N = N;
  g.n = n;
  g.off = off < 0 ? -1 : 1;
  g.tg = tile_geom(N, kWsR);
  WsGeom gi = g, ge = g;
  gi.tiles = tile_count(g.tg, true);
  ws_chunks(gi, blocks);
  k_residual_ws<FMODE, true><<<blocks, kWsThreads, 0, s>>>(gi, A, part);
  ge.tiles = tile_count(g.tg, false);
  ws_chunks(ge, blocks_edge);
  k_residual_ws<FMODE, false><<<blocks_edge, kWsThreads, 0, s>>>(ge, A, part + 2 * blocks);
}

// ---------------------------------------------------------------------------------------
// The residual of the shifted systems of eq. (2) for the refined solves, as warp tiles:
//   r_j = b_j - lam_j z_j - (kappa/h^2)(4 z_j - sum of the 4 neighbours of z_j),
// complex, z_j and b_j in FP64; output in FP32 times sc_j oscale (sc_j the power of two
// keeping shift j's FP32 right-hand side near unit size, oscale the scaling of the level-0
// right-hand side) with the sums of |sc_j r|^2.  The arithmetic is that of the residual of
// eq. (1) above, per complex component.  A warp tile is 30 output columns (lanes
// 1..30) by kSwR rows of one shift; each complex component has its own fixed-point scale
// (warp max of the tile's exponents), its exact stencil difference in three FP32 limbs,
// and z itself in the tile's units from the limbs; lam_j z_j and the sums are float-float
// with the constants scaled to those units.  The real and imaginary components are the
// two components of the packed FP32x2 operations.  The next tile's z is loaded while the
// current one is computed.  Interior tiles (every row and column read inside the grid)
// and edge tiles are two kernels, compiled apart; in each, CTA x of shift j takes that
// kernel's tiles x, x + gx, ... (one per warp); frozen shifts get a zero right-hand side
// and no sums.
constexpr int kSwR = 4;

template <bool FULL>
__global__ void __launch_bounds__(kWsThreads, 2)
k_shift_residual_ws(int N, const double2 *__restrict__ z, const double2 *__restrict__ b,
                    const double2 *__restrict__ lam, double off, float oscale,
                    const float *__restrict__ sc, View out, const int *__restrict__ frozen,
                    double *__restrict__ part, int pstride, int poff) {
  constexpr int R = kSwR;
  __shared__ float2 red[kWsWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.y;
  const long long m = (long long)N * N;
  const TileGeom g = tile_geom(N, R);
  const int tiles = tile_count(g, FULL);
  float2 *o = reinterpret_cast<float2 *>(out.p) + (long long)j * out.plane;
  double *pj = part + (long long)j * pstride + poff + blockIdx.x;
  const int t_first = blockIdx.x * kWsWarps + warp, t_step = gridDim.x * kWsWarps;
  if (frozen && frozen[j]) {
    for (int t = t_first; t < tiles; t += t_step) {
      int by, sx;
      tile_at(g, FULL, t, by, sx);
      const int i0 = by * R, c = sx * kWsOut - 1 + lane;
      if (lane >= 1 && lane <= kWsOut && c < N)
#pragma unroll
        for (int q = 0; q < R; q++)
          if (i0 + q < N) o[(long long)(i0 + q) * out.pitch + c] = make_float2(0.f, 0.f);
    }
    if (threadIdx.x == 0) *pj = 0.0;
    return;
  }
  const double2 *zj = z + (long long)j * m, *bj = b + (long long)j * m;
  const double2 lj = lam[j];
  const DF lr = split(lj.x), li = split(lj.y), offd = split(off);
  const float2 scj = bc2(sc[j]), osc = bc2(oscale);
  DF ar = {0.f, 0.f};
  ulonglong2 raw[R + 2];
  auto load_z = [&](int t) {
    int by, sx;
    tile_at(g, FULL, t, by, sx);
    const int i0 = by * R, c = sx * kWsOut - 1 + lane;
    const bool cin = FULL || (unsigned)c < (unsigned)N;
    const double2 *zc = zj + (long long)(i0 - 1) * N + (cin ? c : 0);
#pragma unroll
    for (int e = 0; e < R + 2; e++) {
      const bool ok = FULL || (cin && (unsigned)(i0 - 1 + e) < (unsigned)N);
      raw[e] = ok ? *reinterpret_cast<const ulonglong2 *>(zc + (long long)e * N) : make_ulonglong2(0ull, 0ull);
    }
  };
  if (t_first < tiles) load_z(t_first);
  for (int t = t_first; t < tiles; t += t_step) {
    int by, sx;
    tile_at(g, FULL, t, by, sx);
    const int i0 = by * R, c = sx * kWsOut - 1 + lane;
    const bool outc = lane >= 1 && lane <= kWsOut && (FULL || c < N);
    const int nr = FULL ? R : min(R, N - i0);
    double2 bq[R];
#pragma unroll
    for (int q = 0; q < R; q++)
      bq[q] = (FULL || (outc && q < nr)) ? bj[(long long)(i0 + q) * N + c] : make_double2(0.0, 0.0);
    // largest exponent of each component over the warp tile, then the limbs (component x:
    // real, y: imaginary)
    unsigned er = 0, ei = 0;
#pragma unroll
    for (int e = 0; e < R + 2; e++) {
      er = max(er, (unsigned)(raw[e].x >> 32) & 0x7FFFFFFFu);
      ei = max(ei, (unsigned)(raw[e].y >> 32) & 0x7FFFFFFFu);
    }
    er = __reduce_max_sync(0xffffffffu, er) >> 20;
    ei = __reduce_max_sync(0xffffffffu, ei) >> 20;
    Limbs2 Q[R + 2];
#pragma unroll
    for (int e = 0; e < R + 2; e++) Q[e] = limbs2(limb_bits(raw[e].x, er), limb_bits(raw[e].y, ei));
    if (t + t_step < tiles) load_z(t + t_step);  // the next tile, while this one is computed
    const bool bad = er > 1081 + 126 || ei > 1081 + 126;
    const int Sr = 1081 - (int)er, Si = 1081 - (int)ei;
    const int sr = Sr > 252 ? 252 : Sr, si = Si > 252 ? 252 : Si;
    // constants in the units of the component they multiply: (lr zr, lr zi), (li zi, -li zr)
    // and off (T1r, T1i)
    const DF qr = df_scale_down(offd, sr), qi = df_scale_down(offd, si);
    const DF lrr = df_scale_down(lr, sr), lri = df_scale_down(lr, si);
    const DF lir = df_scale_down(li, sr), lii = df_scale_down(li, si);
    const DF2 q2 = {make_float2(qr.hi, qi.hi), make_float2(qr.lo, qi.lo)};
    const DF2 l1 = {make_float2(lrr.hi, lri.hi), make_float2(lrr.lo, lri.lo)};
    const DF2 l2 = {make_float2(lii.hi, -lir.hi), make_float2(lii.lo, -lir.lo)};
    const float2 scale = bad ? bc2(__int_as_float(0x7FC00000)) : scj;
    float2 rowr = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < R; q++) {
      // exact stencil differences of both components, as float-float pairs
      const Limbs2 &U = Q[q], &C = Q[q + 1], &D = Q[q + 2];
      const float2 a2 = stencil2(U.l2, C.l2, D.l2);
      const float2 a1 = stencil2(U.l1, C.l1, D.l1);
      const float2 a0 = stencil2(U.l0, C.l0, D.l0);
      DF2 T = two_sum2(a2, a1);
      T.lo = add2(T.lo, a0);
      // z in the tile's units, and with its components swapped
      DF2 Z = fast_two_sum2(C.l2, C.l1);
      Z.lo = add2(Z.lo, C.l0);
      const DF2 Zs = {make_float2(Z.hi.y, Z.hi.x), make_float2(Z.lo.y, Z.lo.x)};
      const DF br = split(bq[q].x), bi = split(bq[q].y);
      const DF2 B2 = {make_float2(br.hi, bi.hi), make_float2(br.lo, bi.lo)};
      // (real, imaginary) = b - (lr zr, lr zi) + (li zi, -li zr) - off (T1r, T1i)
      const DF2 P1 = mul_un2(l1, Z), P2 = mul_un2(l2, Zs), P3 = mul_un2(q2, T);
      const float2 lo = add2(sub2(B2.lo, P1.lo), sub2(P2.lo, P3.lo));
      DF2 s = two_sum2(B2.hi, neg2(P1.hi));
      float2 el = s.lo;
      s = two_sum2(s.hi, P2.hi);
      el = add2(el, s.lo);
      s = two_sum2(s.hi, neg2(P3.hi));
      el = add2(el, s.lo);
      const float2 rv = mul2(add2(s.hi, add2(lo, el)), scale);
      if (outc && q < nr) {
        o[(long long)(i0 + q) * out.pitch + c] = mul2(rv, osc);
        rowr = fma2(rv, rv, rowr);
      }
    }
    ar = df_add(ar, DF{__fadd_rn(rowr.x, rowr.y), 0.f});
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) ar = df_add(ar, df_shfl_down(ar, o2));
  if (lane == 0) red[warp] = make_float2(ar.hi, ar.lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    DF s0 = {0.f, 0.f};
    for (int w = 0; w < kWsWarps; w++) s0 = df_add(s0, DF{red[w].x, red[w].y});
    *pj = (double)s0.hi + (double)s0.lo;
  }
}

}  // namespace

// two CTAs per SM for the interior tiles, two per SM for the edge tiles
int residual_fx_blocks(int num_sms) { return 4 * num_sms; }

// CTAs per shift of the shifted residuals: about eight waves of two CTAs per SM over all
// shifts (the CTAs of a wave do equal work, so a last partial wave costs at most an
// eighth), but no more CTAs than give each warp one warp tile, nor more than grid rows;
// at least two (the interior and the edge tiles take at least one each)
int shift_residual_blocks(int N, int n, int num_sms) {
  const int want = (16 * num_sms + n - 1) / n;
  const long long tiles = (long long)((N + kWsOut - 1) / kWsOut) * ((N + kSwR - 1) / kSwR);
  const int cap = (int)std::min<long long>(N, (tiles + kWsWarps - 1) / kWsWarps);
  return std::max(2, std::min(want, cap));
}

// gx CTAs per shift, split between the interior and the edge kernels in proportion to their
// tiles (at least one each); part[j gx + x] = the sum of CTA x of shift j, the edge kernel's
// CTAs after the interior kernel's
void launch_shift_residual_fx(cudaStream_t s, int gx, int N, int n, const double2 *z, const double2 *b,
                              const double2 *lam, double off, float oscale, const float *sc, View out,
                              const int *frozen, double *part) {
  const TileGeom g = tile_geom(N, kSwR);
  const double fe = (double)tile_count(g, false) / ((double)g.tx * g.ty);
  const int ge = std::min(gx - 1, std::max(1, (int)std::lround(gx * fe))), gi = gx - ge;
  k_shift_residual_ws<true><<<dim3(gi, n), kWsThreads, 0, s>>>(N, z, b, lam, off, oscale, sc, out, frozen,
                                                               part, gx, 0);
  k_shift_residual_ws<false><<<dim3(ge, n), kWsThreads, 0, s>>>(N, z, b, lam, off, oscale, sc, out, frozen,
                                                                part, gx, gi);
}

void launch_residual_fx(cudaStream_t s, int blocks, int N, int n, int off, float2 ihf, float *r,
                        const double *u, const double *f, const double *u0, const float4 *kbd,
                        const float2 *ku0, float oscale, float fscale, bool want_f, double *part,
                        const float2 *fc_in, float2 *fc_out) {
  const WsArgs A{r, u, f, u0, kbd, ku0, DF{ihf.x, ihf.y}, oscale, fscale, want_f ? 1 : 0, fc_in, fc_out};
  const int be = std::max(1, blocks / 2), bi = std::max(1, blocks - be);
  if (fc_in)
    launch_ws<2>(s, bi, be, N, n, off, A, part);
  else if (fc_out)
    launch_ws<1>(s, bi, be, N, n, off, A, part);
  else
    launch_ws<0>(s, bi, be, N, n, off, A, part);
}

}  // namespace pd
