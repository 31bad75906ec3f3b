// Warp-streaming versions of the two fused multigrid kernels (Sec. 2-3) for the
// global-memory levels:
//
//   k_sr_stream: last pre-smoothing step + residual + full weighting (+ sum |rt|^2)
//       z' = z + omega M rt(z),  bt_c = (1/4)[1 2 1; 2 4 2; 1 2 1] rt(z')
//   k_ps_stream: linear interpolation + correction + first post-smoothing step
//       z'' = z' + P e_c,  z''' = z'' + omega M rt(z'')
//   with rt(z) = bt - (4 + eta) z + (sum of the 4 neighbours of z), bt = h^2 b.
//
// Each warp owns a strip of 64 grid columns (2 per lane; the 56 middle ones are its
// output, 4 on each side are recomputed halo) and streams down a segment of `seg` rows
// (even; chosen per level by the set-up autotuner).
// Horizontal neighbours come from the adjacent lanes by shuffles, vertical ones from
// short register windows of the previous rows, so every input value is read from
// memory once per strip and nothing waits at a CTA barrier.  Rows are prefetched
// kDepth rows ahead with cp.async into a per-warp shared-memory ring (zero-filled
// outside the grid: the homogeneous Dirichlet values of z).  The outermost lanes get
// wrong neighbours from the shuffles; with 4 halo columns on each side those errors
// never reach an output column (each stage spreads them by one column).
#include "cplx.cuh"
#include "pd_internal.h"
#include "tma.cuh"

#include <algorithm>

namespace pd {
namespace {

constexpr int kLanes = 32;
constexpr int kStripOut = 56;     // output columns per warp strip
constexpr int kDepth = 4;         // rows prefetched ahead
constexpr int kWarpsPerCta = 8;

// 2 consecutive complex values of one lane
template <typename C> struct Pair {
  C v[2];
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename C> __device__ __forceinline__ C shfl_up1(C x) {
  C r;
  r.x = __shfl_up_sync(0xffffffffu, x.x, 1);
  r.y = __shfl_up_sync(0xffffffffu, x.y, 1);
  return r;
}
template <typename C> __device__ __forceinline__ C shfl_dn1(C x) {
  C r;
  r.x = __shfl_down_sync(0xffffffffu, x.x, 1);
  r.y = __shfl_down_sync(0xffffffffu, x.y, 1);
  return r;
}
template <typename C> __device__ __forceinline__ C sel(bool keep, C x) {
  return keep ? x : czero<C>();
}

// copies the lane's two complex values of row `row`, columns a, a+1, of shift plane
// `base` into shared memory; zeros outside the grid (rows, or a pair wholly outside)
// IN: the caller guarantees row and both columns inside the grid (no predicates)
template <typename C, bool IN = false>
__device__ __forceinline__ void load_pair(uint32_t dst, const C *base, long long pitch, int N, int row,
                                          int a) {
  const bool ok = IN || ((unsigned)row < (unsigned)N && a >= 0 && a < N);
  // zero fill outside the grid from the nearest pair inside it (zero-fill copies still send
  // their source address; one shared address per plane would become a hot spot)
  const C *src = base + (IN ? (long long)row * pitch + a
                            : (long long)min(max(row, 0), N - 1) * pitch + min(max(a, 0), (N - 1) & ~1));
  if (sizeof(C) == 8) {
    cp_async16(dst, src, ok ? 16 : 0);  // a+1 may be the padding column: masked on use
  } else {
    cp_async16(dst, src, ok ? 16 : 0);
    cp_async16(dst + 16, src + 1, (IN || (ok && a + 1 < N)) ? 16 : 0);
  }
}

// A unit (strip x segment of one shift) whose loaded rows and columns, coarse rows and
// columns included, all lie inside the grid: its boundary tests fold away.
__device__ __forceinline__ bool interior_unit(int N, int x0, int y0, int y1) {
  return x0 >= 4 && x0 + 61 <= N && y0 >= 4 && y1 + 4 <= N;
}

template <typename C> __device__ __forceinline__ Pair<C> read_pair(const C *s) {
  Pair<C> p;
  p.v[0] = s[0];
  p.v[1] = s[1];
  return p;
}

// one unit of k_sr_stream (see above); IN: interior_unit
template <typename T, bool ZZERO, bool NORM, bool IN>
__device__ __forceinline__ void sr_unit(int N, int seg, int u, int nsx, int nsy, int Nc, int lane,
                                        typename Cx<T>::type *ring, const View &z, const View &b,
                                        const View &zout, const View &bc,
                                        const Coef<T> *__restrict__ coef,
                                        double *__restrict__ partials, int part_stride) {
  using C = typename Cx<T>::type;
  const int sx = u % nsx, sy = (u / nsx) % nsy, j = u / (nsx * nsy);
  const Coef<T> cf = coef[j];
  const int x0 = sx * kStripOut, y0 = sy * seg, y1 = min(y0 + seg, N);
  const int xend = min(x0 + kStripOut, N);
  const int a = x0 - 4 + 2 * lane;  // this lane's columns a, a+1
  const bool cin0 = IN || (a >= 0 && a < N), cin1 = IN || (a + 1 >= 0 && a + 1 < N);
  const bool out0 = a >= x0 && a < xend, out1 = a + 1 >= x0 && a + 1 < xend;
  const C *zb = reinterpret_cast<const C *>(z.p) + (long long)j * z.plane;
  const C *bb = reinterpret_cast<const C *>(b.p) + (long long)j * b.plane;
  C *zo = reinterpret_cast<C *>(zout.p) + (long long)j * zout.plane;
  C *bco = reinterpret_cast<C *>(bc.p) + (long long)j * bc.plane;
  const int L = y1 - y0 + 7;  // rows y0-3 .. y1+3
  auto slot_z = [&](int s) { return ring + ((s % kDepth) * 2 + 0) * kLanes * 2 + lane * 2; };
  auto slot_b = [&](int s) { return ring + ((s % kDepth) * 2 + 1) * kLanes * 2 + lane * 2; };
  auto issue = [&](int s) {
    if (s < L) {
      const int row = y0 - 3 + s;
      if (!ZZERO) load_pair<C, IN>(smem_u32(slot_z(s)), zb, z.pitch, N, row, a);
      load_pair<C, IN>(smem_u32(slot_b(s)), bb, b.pitch, N, row, a);
    }
    cp_commit();
  };
#pragma unroll
  for (int s = 0; s < kDepth; s++) issue(s);
  // register windows (rows relative to the row i being loaded)
  C zm2[2], zm1[2], bm1[2], bm2[2], bm3[2];
  C rm3[4], rm2[4], rm1[4], zpm4[4], zpm3[4], zpm2[4];
  C va[2];  // vertical 1-2-1 sums of rt(z') of the coarse row being built (own columns)
  va[0] = va[1] = czero<C>();
#pragma unroll
  for (int q = 0; q < 4; q++) {
    rm3[q] = rm2[q] = rm1[q] = zpm4[q] = zpm3[q] = zpm2[q] = czero<C>();
    if (q < 2) zm2[q] = zm1[q] = bm1[q] = bm2[q] = bm3[q] = czero<C>();
  }
  T acc = 0;
#pragma unroll 3
  for (int s = 0; s < L; s++) {
    const int i = y0 - 3 + s;
    cp_wait<kDepth - 1>();
    C zi[2], bi[2];
    {
      const Pair<C> pb = read_pair(slot_b(s));
      bi[0] = pb.v[0];
      bi[1] = sel(cin1, pb.v[1]);
      if (ZZERO) {
        zi[0] = zi[1] = czero<C>();
      } else {
        const Pair<C> pz = read_pair(slot_z(s));
        zi[0] = pz.v[0];
        zi[1] = sel(cin1, pz.v[1]);
      }
    }
    issue(s + kDepth);
    // rt of z on row i-1
    const bool r_in = IN || (unsigned)(i - 1) < (unsigned)N;
    C rn[4];
    {
      const C zL = shfl_up1(zm1[1]), zR = shfl_dn1(zm1[0]);
      C r0 = bm1[0], r1 = bm1[1];
      if (!ZZERO) {
        r0 = csub(cadd(r0, cadd(cadd(zm2[0], zi[0]), cadd(zL, zm1[1]))), cmul(cf.d, zm1[0]));
        r1 = csub(cadd(r1, cadd(cadd(zm2[1], zi[1]), cadd(zm1[0], zR))), cmul(cf.d, zm1[1]));
      }
      r0 = sel(r_in && cin0, r0);
      r1 = sel(r_in && cin1, r1);
      if (NORM && i - 1 >= y0 && i - 1 < y1) {
        if (out0) acc += r0.x * r0.x + r0.y * r0.y;
        if (out1) acc += r1.x * r1.x + r1.y * r1.y;
      }
      rn[0] = shfl_up1(r1);
      rn[1] = r0;
      rn[2] = r1;
      rn[3] = shfl_dn1(r0);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      rm3[q] = rm2[q];
      rm2[q] = rm1[q];
      rm1[q] = rn[q];
    }
    // z' = z + omega M rt on row i-2
    const bool p_in = IN || (unsigned)(i - 2) < (unsigned)N;
    C zp[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const C e = cadd(cadd(rm3[k + 1], rm1[k + 1]), cadd(rm2[k], rm2[k + 2]));
      const C co = cadd(cadd(rm3[k], rm3[k + 2]), cadd(rm1[k], rm1[k + 2]));
      C upd = cmul(cf.ca, rm2[k + 1]);
      upd = cfma(cf.cb, e, upd);
      upd = cfma(cf.cc, co, upd);
      zp[k] = sel(p_in && (k ? cin1 : cin0), ZZERO ? upd : cadd(zm2[k], upd));
    }
    if (i - 2 >= y0 && i - 2 < y1) {
      C *dst = zo + (long long)(i - 2) * zout.pitch + a;
      if (out0) dst[0] = zp[0];
      if (out1) dst[1] = zp[1];
    }
    {
      const C l = shfl_up1(zp[1]), r = shfl_dn1(zp[0]);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        zpm4[q] = zpm3[q];
        zpm3[q] = zpm2[q];
      }
      zpm2[0] = l;
      zpm2[1] = zp[0];
      zpm2[2] = zp[1];
      zpm2[3] = r;
    }
    // rt of z' on row i-3
    const bool q_in = IN || (unsigned)(i - 3) < (unsigned)N;
    C rp[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const C nb = cadd(cadd(zpm4[k + 1], zpm2[k + 1]), cadd(zpm3[k], zpm3[k + 2]));
      rp[k] = sel(q_in && (k ? cin1 : cin0), csub(cadd(bm3[k], nb), cmul(cf.d, zpm3[k + 1])));
    }
    // full weighting, separable: the vertical 1-2-1 sums per column are accumulated as the
    // rows of rt(z') arrive (row q = i-3: weight 2 on an odd row, the centre of a coarse
    // row; an even row closes the sums of the coarse row centred on q-1 and opens the
    // next), then combined 1-2-1 across the columns a, a+1, a+2 (the last from the right
    // lane) for the coarse point (I, J) at fine (q-1, a+1)
    if (!(i & 1)) {
      va[0] = cadd(va[0], cscale(rp[0], (T)2));
      va[1] = cadd(va[1], cscale(rp[1], (T)2));
    } else {
      va[0] = cadd(va[0], rp[0]);
      va[1] = cadd(va[1], rp[1]);
      const C vr = shfl_dn1(va[0]);
      const int cr = i - 4;
      if (cr >= y0 && cr < y1 && out1) {
        const int I = (cr - 1) >> 1, J = a >> 1;
        if (IN || (I < Nc && J < Nc))
          bco[(long long)I * bc.pitch + J] =
              cscale(cadd(cadd(va[0], vr), cscale(va[1], (T)2)), (T)0.25);
      }
      va[0] = rp[0];
      va[1] = rp[1];
    }
    zm2[0] = zm1[0];
    zm2[1] = zm1[1];
    zm1[0] = zi[0];
    zm1[1] = zi[1];
    bm3[0] = bm2[0];
    bm3[1] = bm2[1];
    bm2[0] = bm1[0];
    bm2[1] = bm1[1];
    bm1[0] = bi[0];
    bm1[1] = bi[1];
  }
  cp_wait<0>();
  if (NORM) {
    double s = (double)acc;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) partials[(long long)j * part_stride + sy * nsx + sx] = s;
  }
}

template <typename T, bool ZZERO, bool NORM>
__global__ void __launch_bounds__(kWarpsPerCta * kLanes, sizeof(T) == 4 ? 2 : 1)
k_sr_stream(int N, int n, int seg, View z, View b, View zout, View bc,
            const Coef<T> *__restrict__ coef, const int *__restrict__ active,
            double *__restrict__ partials, int part_stride) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char ring_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // ring: kDepth slots x (z row, bt row) x 32 lanes x 2 complex
  C *ring = reinterpret_cast<C *>(ring_raw) + (size_t)wib * kDepth * 2 * kLanes * 2;
  const int nsx = (N + kStripOut - 1) / kStripOut, nsy = (N + seg - 1) / seg;
  const int total = n * nsx * nsy;
  const int Nc = (N - 1) / 2;
  const int gw = blockIdx.x * kWarpsPerCta + wib, nw = gridDim.x * kWarpsPerCta;
  for (int u = gw; u < total; u += nw) {
    const int sx = u % nsx, sy = (u / nsx) % nsy, j = u / (nsx * nsy);
    if (active && !active[j]) continue;
    const int x0 = sx * kStripOut, y0 = sy * seg, y1 = min(y0 + seg, N);
    if (interior_unit(N, x0, y0, y1))
      sr_unit<T, ZZERO, NORM, true>(N, seg, u, nsx, nsy, Nc, lane, ring, z, b, zout, bc, coef,
                                    partials, part_stride);
    else
      sr_unit<T, ZZERO, NORM, false>(N, seg, u, nsx, nsy, Nc, lane, ring, z, b, zout, bc, coef,
                                     partials, part_stride);
  }
}

// one unit of k_ps_stream (see above); IN: interior_unit
template <typename T, bool IN>
__device__ __forceinline__ void ps_unit(int N, int seg, int u, int nsx, int nsy, int Nc, int lane,
                                        typename Cx<T>::type *ring, const View &z, const View &e,
                                        const View &b, const View &zout,
                                        const Coef<T> *__restrict__ coef) {
  using C = typename Cx<T>::type;
  const int sx = u % nsx, sy = (u / nsx) % nsy, j = u / (nsx * nsy);
  const Coef<T> cf = coef[j];
  const int x0 = sx * kStripOut, y0 = sy * seg, y1 = min(y0 + seg, N);
  const int xend = min(x0 + kStripOut, N);
  const int a = x0 - 4 + 2 * lane;
  const int J = a >> 1;  // coarse column of the odd fine column a+1
  const bool cin0 = IN || (a >= 0 && a < N), cin1 = IN || (a + 1 >= 0 && a + 1 < N);
  const bool out0 = a >= x0 && a < xend, out1 = a + 1 >= x0 && a + 1 < xend;
  const C *zb = reinterpret_cast<const C *>(z.p) + (long long)j * z.plane;
  const C *eb = reinterpret_cast<const C *>(e.p) + (long long)j * e.plane;
  const C *bb = reinterpret_cast<const C *>(b.p) + (long long)j * b.plane;
  C *zo = reinterpret_cast<C *>(zout.p) + (long long)j * zout.plane;
  const int L = y1 - y0 + 4;  // rows y0-2 .. y1+1
  auto slot = [&](int s, int k) { return ring + ((s % kDepth) * 3 + k) * kLanes * 2 + lane * 2; };
  // coarse row m (complex at column J) into the slot's third row; zero outside
  auto load_coarse = [&](uint32_t dst, int m) {
    const bool ok = IN || ((unsigned)m < (unsigned)Nc && (unsigned)J < (unsigned)Nc);
    const C *src = eb + (IN ? (long long)m * e.pitch + J
                            : (long long)min(max(m, 0), Nc - 1) * e.pitch + min(max(J, 0), Nc - 1));
    if (sizeof(C) == 8) cp_async8(dst, src, ok ? 8 : 0);
    else cp_async16(dst, src, ok ? 16 : 0);
  };
  auto issue = [&](int s) {
    if (s < L) {
      const int row = y0 - 2 + s;
      load_pair<C, IN>(smem_u32(slot(s, 0)), zb, z.pitch, N, row, a);
      load_pair<C, IN>(smem_u32(slot(s, 1)), bb, b.pitch, N, row, a);
      if (!(row & 1)) load_coarse(smem_u32(slot(s, 2)), row >> 1);  // coarse row m at fine 2m
    }
    cp_commit();
  };
  // coarse row y0/2 - 2: the first fine row y0 - 2 (even) shifts it into eprev and
  // loads row y0/2 - 1 into ecur
  C eprev = czero<C>(), ecur;
  {
    const int m = y0 / 2 - 2;
    const bool ok = IN || ((unsigned)m < (unsigned)Nc && (unsigned)J < (unsigned)Nc);
    ecur = ok ? eb[(long long)m * e.pitch + J] : czero<C>();
  }
#pragma unroll
  for (int s = 0; s < kDepth; s++) issue(s);
  C zz1[4], zz0[4], bm1[2], rm3[4], rm2[4], rm1[4];  // z'' rows i-1 (zz1), i-2 (zz0)
#pragma unroll
  for (int q = 0; q < 4; q++) {
    zz1[q] = zz0[q] = rm3[q] = rm2[q] = rm1[q] = czero<C>();
    if (q < 2) bm1[q] = czero<C>();
  }
#pragma unroll 3
  for (int s = 0; s < L; s++) {
    const int i = y0 - 2 + s;
    cp_wait<kDepth - 1>();
    C zi[2], bi[2];
    {
      const Pair<C> pz = read_pair(slot(s, 0));
      const Pair<C> pb = read_pair(slot(s, 1));
      zi[0] = pz.v[0];
      zi[1] = sel(cin1, pz.v[1]);
      bi[0] = pb.v[0];
      bi[1] = sel(cin1, pb.v[1]);
      if (!(i & 1)) {
        eprev = ecur;
        ecur = *slot(s, 2);
      }
    }
    issue(s + kDepth);
    // z'' = z' + P e_c on row i: odd rows sit on coarse row (i-1)/2 = ecur, even rows
    // between eprev (i/2 - 1) and ecur (i/2); odd columns on coarse column J, even
    // columns between J-1 (from the left lane) and J
    const bool i_in = IN || (unsigned)i < (unsigned)N;
    C zn[4];
    {
      const C ev = (i & 1) ? ecur : cscale(cadd(eprev, ecur), (T)0.5);
      const C evl = shfl_up1(ev);
      const C p0 = cscale(cadd(evl, ev), (T)0.5), p1 = ev;
      const C z0 = sel(i_in && cin0, cadd(zi[0], p0));
      const C z1 = sel(i_in && cin1, cadd(zi[1], p1));
      zn[0] = shfl_up1(z1);
      zn[1] = z0;
      zn[2] = z1;
      zn[3] = shfl_dn1(z0);
    }
    // rt of z'' on row i-1
    const bool r_in = IN || (unsigned)(i - 1) < (unsigned)N;
    C rn[4];
    {
      C r0 = csub(cadd(bm1[0], cadd(cadd(zz0[1], zn[1]), cadd(zz1[0], zz1[2]))), cmul(cf.d, zz1[1]));
      C r1 = csub(cadd(bm1[1], cadd(cadd(zz0[2], zn[2]), cadd(zz1[1], zz1[3]))), cmul(cf.d, zz1[2]));
      r0 = sel(r_in && cin0, r0);
      r1 = sel(r_in && cin1, r1);
      rn[0] = shfl_up1(r1);
      rn[1] = r0;
      rn[2] = r1;
      rn[3] = shfl_dn1(r0);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      rm3[q] = rm2[q];
      rm2[q] = rm1[q];
      rm1[q] = rn[q];
    }
    // z''' = z'' + omega M rt on row i-2 (z''(i-2) is zz0 before the shift below)
    if (i - 2 >= y0 && i - 2 < y1) {
      C out[2];
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const C e2 = cadd(cadd(rm3[k + 1], rm1[k + 1]), cadd(rm2[k], rm2[k + 2]));
        const C co = cadd(cadd(rm3[k], rm3[k + 2]), cadd(rm1[k], rm1[k + 2]));
        C upd = cmul(cf.ca, rm2[k + 1]);
        upd = cfma(cf.cb, e2, upd);
        upd = cfma(cf.cc, co, upd);
        out[k] = cadd(zz0[k + 1], upd);
      }
      C *dst = zo + (long long)(i - 2) * zout.pitch + a;
      if (out0) dst[0] = out[0];
      if (out1) dst[1] = out[1];
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      zz0[q] = zz1[q];
      zz1[q] = zn[q];
    }
    bm1[0] = bi[0];
    bm1[1] = bi[1];
  }
  cp_wait<0>();
}

template <typename T>
__global__ void __launch_bounds__(kWarpsPerCta * kLanes, sizeof(T) == 4 ? 2 : 1)
k_ps_stream(int N, int n, int seg, View z, View e, View b, View zout,
            const Coef<T> *__restrict__ coef, const int *__restrict__ active) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char ring_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // ring: kDepth slots x (z' row, bt row, coarse row) x 32 lanes x 2 complex
  C *ring = reinterpret_cast<C *>(ring_raw) + (size_t)wib * kDepth * 3 * kLanes * 2;
  const int nsx = (N + kStripOut - 1) / kStripOut, nsy = (N + seg - 1) / seg;
  const int total = n * nsx * nsy;
  const int Nc = (N - 1) / 2;
  const int gw = blockIdx.x * kWarpsPerCta + wib, nw = gridDim.x * kWarpsPerCta;
  for (int u = gw; u < total; u += nw) {
    const int sx = u % nsx, sy = (u / nsx) % nsy, j = u / (nsx * nsy);
    if (active && !active[j]) continue;
    const int x0 = sx * kStripOut, y0 = sy * seg, y1 = min(y0 + seg, N);
    if (interior_unit(N, x0, y0, y1))
      ps_unit<T, true>(N, seg, u, nsx, nsy, Nc, lane, ring, z, e, b, zout, coef);
    else
      ps_unit<T, false>(N, seg, u, nsx, nsy, Nc, lane, ring, z, e, b, zout, coef);
  }
}

// The same two kernels over the units of several instance-levels in one launch (batches
// of uneven instances): unit u belongs to the task whose range [ubegin, next ubegin)
// holds it.
template <typename T, bool ZZERO, bool NORM>
__global__ void __launch_bounds__(kWarpsPerCta * kLanes, sizeof(T) == 4 ? 2 : 1)
k_sr_multi(const StreamTask<T> *__restrict__ tasks, int ntasks, int total) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char ring_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  C *ring = reinterpret_cast<C *>(ring_raw) + (size_t)wib * kDepth * 2 * kLanes * 2;
  const int gw = blockIdx.x * kWarpsPerCta + wib, nw = gridDim.x * kWarpsPerCta;
  int t = 0;
  for (int u = gw; u < total; u += nw) {
    while (t + 1 < ntasks && u >= tasks[t + 1].ubegin) t++;
    const StreamTask<T> &k = tasks[t];
    const int N = k.N, seg = k.seg, ul = u - k.ubegin;
    const int nsx = (N + kStripOut - 1) / kStripOut, nsy = (N + seg - 1) / seg;
    const int sx = ul % nsx, sy = (ul / nsx) % nsy, j = ul / (nsx * nsy);
    if (k.active && !k.active[j]) continue;
    const int x0 = sx * kStripOut, y0 = sy * seg, y1 = min(y0 + seg, N), Nc = (N - 1) / 2;
    if (interior_unit(N, x0, y0, y1))
      sr_unit<T, ZZERO, NORM, true>(N, seg, ul, nsx, nsy, Nc, lane, ring, k.z, k.b, k.zout, k.x, k.coef,
                                    k.partials, k.part_stride);
    else
      sr_unit<T, ZZERO, NORM, false>(N, seg, ul, nsx, nsy, Nc, lane, ring, k.z, k.b, k.zout, k.x, k.coef,
                                     k.partials, k.part_stride);
  }
}

template <typename T>
__global__ void __launch_bounds__(kWarpsPerCta * kLanes, sizeof(T) == 4 ? 2 : 1)
k_ps_multi(const StreamTask<T> *__restrict__ tasks, int ntasks, int total) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char ring_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  C *ring = reinterpret_cast<C *>(ring_raw) + (size_t)wib * kDepth * 3 * kLanes * 2;
  const int gw = blockIdx.x * kWarpsPerCta + wib, nw = gridDim.x * kWarpsPerCta;
  int t = 0;
  for (int u = gw; u < total; u += nw) {
    while (t + 1 < ntasks && u >= tasks[t + 1].ubegin) t++;
    const StreamTask<T> &k = tasks[t];
    const int N = k.N, seg = k.seg, ul = u - k.ubegin;
    const int nsx = (N + kStripOut - 1) / kStripOut, nsy = (N + seg - 1) / seg;
    const int sx = ul % nsx, sy = (ul / nsx) % nsy, j = ul / (nsx * nsy);
    if (k.active && !k.active[j]) continue;
    const int x0 = sx * kStripOut, y0 = sy * seg, y1 = min(y0 + seg, N), Nc = (N - 1) / 2;
    if (interior_unit(N, x0, y0, y1))
      ps_unit<T, true>(N, seg, ul, nsx, nsy, Nc, lane, ring, k.z, k.x, k.b, k.zout, k.coef);
    else
      ps_unit<T, false>(N, seg, ul, nsx, nsy, Nc, lane, ring, k.z, k.x, k.b, k.zout, k.coef);
  }
}

template <int ROWS> constexpr int ring_bytes(int elem) { return kWarpsPerCta * kDepth * ROWS * kLanes * 2 * elem; }

}  // namespace

int stream_units(int N, int seg) {
  return ((N + kStripOut - 1) / kStripOut) * ((N + seg - 1) / seg);
}

template <typename T>
void launch_sr_stream(cudaStream_t s, int grid, int N, int n, int seg, View z, View b, View zout,
                      View bc, const Coef<T> *coef, const int *active, bool z_zero, double *partials,
                      int part_stride) {
  const int smem = ring_bytes<2>((int)sizeof(typename Cx<T>::type));
  const int th = kWarpsPerCta * kLanes;
  if (z_zero) {
    if (partials)
      k_sr_stream<T, true, true><<<grid, th, smem, s>>>(N, n, seg, z, b, zout, bc, coef, active, partials, part_stride);
    else
      k_sr_stream<T, true, false><<<grid, th, smem, s>>>(N, n, seg, z, b, zout, bc, coef, active, partials, part_stride);
  } else {
    if (partials)
      k_sr_stream<T, false, true><<<grid, th, smem, s>>>(N, n, seg, z, b, zout, bc, coef, active, partials, part_stride);
    else
      k_sr_stream<T, false, false><<<grid, th, smem, s>>>(N, n, seg, z, b, zout, bc, coef, active, partials, part_stride);
  }
}

template <typename T>
void launch_ps_stream(cudaStream_t s, int grid, int N, int n, int seg, View z, View e, View b,
                      View zout, const Coef<T> *coef, const int *active) {
  const int smem = ring_bytes<3>((int)sizeof(typename Cx<T>::type));
  k_ps_stream<T><<<grid, kWarpsPerCta * kLanes, smem, s>>>(N, n, seg, z, e, b, zout, coef, active);
}

template <typename T>
void launch_sr_multi(cudaStream_t s, int grid, const StreamTask<T> *tasks, int ntasks, int total, bool z_zero,
                     bool norm) {
  const int smem = ring_bytes<2>((int)sizeof(typename Cx<T>::type));
  const int th = kWarpsPerCta * kLanes;
  if (z_zero) {
    if (norm) k_sr_multi<T, true, true><<<grid, th, smem, s>>>(tasks, ntasks, total);
    else k_sr_multi<T, true, false><<<grid, th, smem, s>>>(tasks, ntasks, total);
  } else {
    if (norm) k_sr_multi<T, false, true><<<grid, th, smem, s>>>(tasks, ntasks, total);
    else k_sr_multi<T, false, false><<<grid, th, smem, s>>>(tasks, ntasks, total);
  }
}

template <typename T>
void launch_ps_multi(cudaStream_t s, int grid, const StreamTask<T> *tasks, int ntasks, int total) {
  const int smem = ring_bytes<3>((int)sizeof(typename Cx<T>::type));
  k_ps_multi<T><<<grid, kWarpsPerCta * kLanes, smem, s>>>(tasks, ntasks, total);
}

template <typename T> cudaError_t prepare_stream() {
  const int a = ring_bytes<2>((int)sizeof(typename Cx<T>::type));
  const int b = ring_bytes<3>((int)sizeof(typename Cx<T>::type));
  cudaError_t e;
#define PD_ATTR(K, S)                                                                  \
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, S);         \
  if (e != cudaSuccess) return e;
  PD_ATTR((k_sr_stream<T, false, false>), a)
  PD_ATTR((k_sr_stream<T, false, true>), a)
  PD_ATTR((k_sr_stream<T, true, false>), a)
  PD_ATTR((k_sr_stream<T, true, true>), a)
  PD_ATTR((k_ps_stream<T>), b)
  PD_ATTR((k_sr_multi<T, false, false>), a)
  PD_ATTR((k_sr_multi<T, false, true>), a)
  PD_ATTR((k_sr_multi<T, true, false>), a)
  PD_ATTR((k_sr_multi<T, true, true>), a)
  PD_ATTR((k_ps_multi<T>), b)
#undef PD_ATTR
  return cudaSuccess;
}

template <typename T> int stream_grid(int num_sms) {
  // resident CTAs per SM from the occupancy calculator, times the SMs
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_sr_stream<T, false, false>, kWarpsPerCta * kLanes,
                                                ring_bytes<2>((int)sizeof(typename Cx<T>::type)));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ps_stream<T>, kWarpsPerCta * kLanes,
                                                ring_bytes<3>((int)sizeof(typename Cx<T>::type)));
  const int per = std::max(1, std::min(a, b));
  return per * num_sms;
}

#define PD_INST_S(T)                                                                             \
  template void launch_sr_stream<T>(cudaStream_t, int, int, int, int, View, View, View, View,   \
                                    const Coef<T> *, const int *, bool, double *, int);          \
  template void launch_ps_stream<T>(cudaStream_t, int, int, int, int, View, View, View, View,   \
                                    const Coef<T> *, const int *);                               \
  template void launch_sr_multi<T>(cudaStream_t, int, const StreamTask<T> *, int, int, bool, bool); \
  template void launch_ps_multi<T>(cudaStream_t, int, const StreamTask<T> *, int, int);          \
  template int stream_grid<T>(int);                                                              \
  template cudaError_t prepare_stream<T>();

PD_INST_S(float)
PD_INST_S(double)

}  // namespace pd
