// Fused, persistent multigrid kernels for the global-memory levels (Sec. 2-3), with
// TMA-staged, double-buffered tiles:
//
//   k_smooth_restrict (last pre-smoothing step + residual + full weighting):
//     z' = z + omega M (bt - h^2 L z),  bt_c = 4 FW(bt - h^2 L z')   [+ sum |rt|^2 of z]
//     reads z, bt once and writes z', bt_c: 3.25 words per fine point instead of the
//     5.25 of separate smoothing and restriction kernels.
//   k_prolong_smooth (linear interpolation + correction + first post-smoothing step):
//     z'' = z' + P e_c,  z''' = z'' + omega M (bt - h^2 L z'')
//     reads z', e_c, bt and writes z''': 3.25 words per point instead of 5.25.
//
// One CTA per SM loops over the tiles of all active shifts; thread 0 issues the TMA
// loads of the next tile (boxes with halos, zero-filled outside the grid, which is the
// homogeneous Dirichlet extension of z) while the CTA computes the current one in
// shared memory.  Every halo value is recomputed locally, so no tile waits on another.
// All waits are bounded: a wait that runs out sets bit 1 of *errflag and the kernel
// leaves after its own copies in flight have landed (bounded as well).
#include <cuda.h>

#include "cplx.cuh"
#include "pd_internal.h"
#include "tma.cuh"

namespace pd {

namespace {

template <typename T> struct FT;
template <> struct FT<float> { static constexpr int TX = 128, TY = 16; };
template <> struct FT<double> { static constexpr int TX = 64, TY = 16; };
constexpr int kFT = 1024;

// TMA x coordinates count 8-byte elements: one per FP32 complex, two per FP64 complex
template <typename T> struct XS { static constexpr int v = sizeof(typename Cx<T>::type) / 8; };

__host__ __device__ constexpr int align128(int b) { return (b + 127) & ~127; }

template <typename C>
__device__ __forceinline__ void stv(const View &v, int j, long long i, long long c, C x) {
  reinterpret_cast<C *>(v.p)[j * v.plane + i * v.pitch + c] = x;
}

// first tile index >= t (stepping by stride) whose shift is still active
__device__ __forceinline__ int next_tile(int t, int stride, int total, int tps, const int *active) {
  while (t < total && active && !active[t / tps]) t += stride;
  return t;
}

template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < NT / 32; k++) s += red[k];
  return s;
}

template <typename T> struct SRLayout {
  using C = typename Cx<T>::type;
  static constexpr int TX = FT<T>::TX, TY = FT<T>::TY;
  // rt(z') is needed on rows/cols [y0, y0+TY] for the coarse points of the tile, so z'
  // on [y0-1, y0+TY+1], rt(z) on [y0-2, y0+TY+2] and z on [y0-3, y0+TY+3]; boxes start
  // at even x (16-byte TMA rule) and have even widths
  static constexpr int ZW = TX + 8, ZH = TY + 7;  // z box: cols x0-4.., rows y0-3..
  static constexpr int BW = TX + 6, BH = TY + 5;  // bt box: cols x0-2.., rows y0-2..
  static constexpr int RW = TX + 5, RH = TY + 5;  // rt: cols x0-2.., rows y0-2..
  static constexpr int PW = TX + 3, PH = TY + 3;  // z': cols x0-1.., rows y0-1..
  static constexpr int QW = TX + 1, QH = TY + 1;  // rt(z'): cols x0.., rows y0.. (in rt's place)
  static constexpr int ZB = align128(ZW * ZH * (int)sizeof(C));
  static constexpr int BB = align128(BW * BH * (int)sizeof(C));
  static constexpr int STAGE = ZB + BB;
  static constexpr int RB = align128(RW * RH * (int)sizeof(C));
  static constexpr int PB = align128(PW * PH * (int)sizeof(C));
  static constexpr int SMEM = 2 * STAGE + RB + PB + 128;  // + alignment slack
};

template <typename T, bool ZZERO, bool NORM>
__global__ void __launch_bounds__(kFT, 1)
k_smooth_restrict(const __grid_constant__ CUtensorMap zmap, const __grid_constant__ CUtensorMap bmap,
                  int N, int n, View zout, View bc, const Coef<T> *__restrict__ coef,
                  const int *__restrict__ active, double *__restrict__ partials, int part_stride,
                  int *__restrict__ errflag) {
  using C = typename Cx<T>::type;
  using Ly = SRLayout<T>;
  constexpr int TX = Ly::TX, TY = Ly::TY;
  constexpr int ZW = Ly::ZW, BW = Ly::BW, RW = Ly::RW, RH = Ly::RH, PW = Ly::PW, PH = Ly::PH;
  constexpr int QW = Ly::QW, QH = Ly::QH;
  constexpr uint32_t TXB = (ZZERO ? 0u : (uint32_t)(Ly::ZW * Ly::ZH * sizeof(C))) +
                           (uint32_t)(Ly::BW * Ly::BH * sizeof(C));
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  __shared__ uint64_t bars[2];
  __shared__ double red[kFT / 32];
  C *R = reinterpret_cast<C *>(smem + 2 * Ly::STAGE);
  C *ZP = reinterpret_cast<C *>(smem + 2 * Ly::STAGE + Ly::RB);
  C *Q = R;
  const int tiles_x = (N + TX - 1) / TX, tiles_y = (N + TY - 1) / TY;
  const int tps = tiles_x * tiles_y, total = n * tps, G = gridDim.x;
  const int Nc = (N - 1) / 2;
  const int tid = threadIdx.x;
  if (tid == 0) {
    prefetch_tensormap(&bmap);
    if (!ZZERO) prefetch_tensormap(&zmap);
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  bool pend[2] = {false, false};  // thread 0: loads in flight per stage
  auto issue = [&](int tt, int s) {
    const int j = tt / tps, tile = tt - j * tps;
    const int y0 = (tile / tiles_x) * TY, x0 = (tile % tiles_x) * TX;
    unsigned char *st = smem + s * Ly::STAGE;
    mbar_arrive_expect_tx(&bars[s], TXB);
    if (!ZZERO) tma_load_3d(st, &zmap, (x0 - 4) * XS<T>::v, y0 - 3, j, &bars[s]);
    tma_load_3d(st + Ly::ZB, &bmap, (x0 - 2) * XS<T>::v, y0 - 2, j, &bars[s]);
    pend[s] = true;
  };
  int t = next_tile(blockIdx.x, G, total, tps, active);
  if (tid == 0 && t < total) issue(t, 0);
  int k = 0;
  for (; t < total; k++) {
    const int s = k & 1;
    const int tn = next_tile(t + G, G, total, tps, active);
    if (tid == 0 && tn < total) {
      fence_proxy_async_smem();
      issue(tn, s ^ 1);
    }
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k >> 1) & 1));
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(errflag, 2);
      break;
    }
    if (tid == 0) pend[s] = false;
    const int j = t / tps, tile = t - j * tps;
    const int y0 = (tile / tiles_x) * TY, x0 = (tile % tiles_x) * TX;
    const C *Zs = reinterpret_cast<const C *>(smem + s * Ly::STAGE);
    const C *Bs = reinterpret_cast<const C *>(smem + s * Ly::STAGE + Ly::ZB);
    const Coef<T> cf = coef[j];
    // phase 1: rt of z on rows y0-2.., cols x0-2.. (zero outside the interior)
    T acc = 0;
    for (int q = tid; q < RH * RW; q += kFT) {
      const int rr = q / RW, cc = q - rr * RW;
      const int i = y0 - 2 + rr, c = x0 - 2 + cc;
      C r = czero<C>();
      if ((unsigned)i < (unsigned)N && (unsigned)c < (unsigned)N) {
        r = Bs[rr * BW + cc];
        if (!ZZERO) {
          const C *zc = &Zs[(rr + 1) * ZW + cc + 2];
          r = csub(cadd(r, cadd(cadd(zc[-ZW], zc[ZW]), cadd(zc[-1], zc[1]))), cmul(cf.d, zc[0]));
        }
        if (NORM && rr >= 2 && rr < TY + 2 && cc >= 2 && cc < TX + 2) acc += r.x * r.x + r.y * r.y;
      }
      R[q] = r;
    }
    __syncthreads();
    // phase 2: z' = z + omega M rt on rows y0-1.., cols x0-1..; the tile itself is stored
    for (int q = tid; q < PH * PW; q += kFT) {
      const int pr = q / PW, pc = q - pr * PW;
      const int i = y0 - 1 + pr, c = x0 - 1 + pc;
      C v = czero<C>();
      if ((unsigned)i < (unsigned)N && (unsigned)c < (unsigned)N) {
        const C *rc = &R[(pr + 1) * RW + pc + 1];
        C upd = cmul(cf.ca, rc[0]);
        const C e = cadd(cadd(rc[-RW], rc[RW]), cadd(rc[-1], rc[1]));
        const C kk = cadd(cadd(rc[-RW - 1], rc[-RW + 1]), cadd(rc[RW - 1], rc[RW + 1]));
        upd = cfma(cf.cb, e, upd);
        upd = cfma(cf.cc, kk, upd);
        v = ZZERO ? upd : cadd(Zs[(pr + 2) * ZW + pc + 3], upd);
        if (pr >= 1 && pr <= TY && pc >= 1 && pc <= TX) stv<C>(zout, j, i, c, v);
      }
      ZP[q] = v;
    }
    __syncthreads();
    // phase 3: rt of z' on rows y0.., cols x0.. (stored where rt of z was)
    for (int q = tid; q < QH * QW; q += kFT) {
      const int qr = q / QW, qc = q - qr * QW;
      const int i = y0 + qr, c = x0 + qc;
      C r = czero<C>();
      if (i < N && c < N) {
        const C *zc = &ZP[(qr + 1) * PW + qc + 1];
        r = csub(cadd(Bs[(qr + 2) * BW + qc + 2], cadd(cadd(zc[-PW], zc[PW]), cadd(zc[-1], zc[1]))),
                 cmul(cf.d, zc[0]));
      }
      Q[q] = r;
    }
    __syncthreads();
    // phase 4: bt_c = (1/4) [1 2 1; 2 4 2; 1 2 1] rt(z') around (2I+1, 2J+1)
    for (int q = tid; q < (TY / 2) * (TX / 2); q += kFT) {
      const int a = q / (TX / 2), b = q - a * (TX / 2);
      const int I = y0 / 2 + a, J = x0 / 2 + b;
      if (I < Nc && J < Nc) {
        const C *rc = &Q[(2 * a + 1) * QW + 2 * b + 1];
        const C e = cadd(cadd(rc[-QW], rc[QW]), cadd(rc[-1], rc[1]));
        const C kk = cadd(cadd(rc[-QW - 1], rc[-QW + 1]), cadd(rc[QW - 1], rc[QW + 1]));
        const C sum = cadd(cadd(cscale(rc[0], (T)4), cscale(e, (T)2)), kk);
        stv<C>(bc, j, I, J, cscale(sum, (T)0.25));
      }
    }
    if (NORM) {
      const double sum = block_sum_d<kFT>((double)acc, red);
      if (tid == 0) partials[(long long)j * part_stride + tile] = sum;
    }
    fence_proxy_async_smem();
    __syncthreads();
    t = tn;
  }
  // a wait that ran out: let this CTA's copies in flight land before leaving
  if (tid == 0)
    for (int s = 0; s < 2; s++)
      if (pend[s]) mbar_wait_bounded(&bars[s], (uint32_t)(((k + (s != (k & 1))) >> 1) & 1));
}

template <typename T> struct PSLayout {
  using C = typename Cx<T>::type;
  static constexpr int TX = FT<T>::TX, TY = FT<T>::TY;
  static constexpr int ZW = TX + 4, ZH = TY + 4;          // z' box: cols x0-2.., rows y0-2..
  static constexpr int EW = TX / 2 + 4, EH = TY / 2 + 3;  // e_c box: x0/2-2.., y0/2-2..
  static constexpr int BW = TX + 4, BH = TY + 2;          // bt box: cols x0-2.., rows y0-1..
  static constexpr int RW = TX + 2, RH = TY + 2;          // rt: cols x0-1.., rows y0-1..
  static constexpr int ZB = align128(ZW * ZH * (int)sizeof(C));
  static constexpr int EB = align128(EW * EH * (int)sizeof(C));
  static constexpr int BB = align128(BW * BH * (int)sizeof(C));
  static constexpr int STAGE = ZB + EB + BB;
  static constexpr int RB = align128(RW * RH * (int)sizeof(C));
  static constexpr int SMEM = 2 * STAGE + RB + 128;  // + alignment slack
};

template <typename T>
__global__ void __launch_bounds__(kFT, 1)
k_prolong_smooth(const __grid_constant__ CUtensorMap zmap, const __grid_constant__ CUtensorMap emap,
                 const __grid_constant__ CUtensorMap bmap, int N, int n, View zout,
                 const Coef<T> *__restrict__ coef, const int *__restrict__ active,
                 int *__restrict__ errflag) {
  using C = typename Cx<T>::type;
  using Ly = PSLayout<T>;
  constexpr int TX = Ly::TX, TY = Ly::TY;
  constexpr int ZW = Ly::ZW, ZH = Ly::ZH, EW = Ly::EW, BW = Ly::BW, RW = Ly::RW, RH = Ly::RH;
  constexpr uint32_t TXB = (uint32_t)((Ly::ZW * Ly::ZH + Ly::EW * Ly::EH + Ly::BW * Ly::BH) * sizeof(C));
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  __shared__ uint64_t bars[2];
  C *R = reinterpret_cast<C *>(smem + 2 * Ly::STAGE);
  const int tiles_x = (N + TX - 1) / TX, tiles_y = (N + TY - 1) / TY;
  const int tps = tiles_x * tiles_y, total = n * tps, G = gridDim.x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    prefetch_tensormap(&zmap);
    prefetch_tensormap(&emap);
    prefetch_tensormap(&bmap);
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  bool pend[2] = {false, false};
  auto issue = [&](int tt, int s) {
    const int j = tt / tps, tile = tt - j * tps;
    const int y0 = (tile / tiles_x) * TY, x0 = (tile % tiles_x) * TX;
    unsigned char *st = smem + s * Ly::STAGE;
    mbar_arrive_expect_tx(&bars[s], TXB);
    tma_load_3d(st, &zmap, (x0 - 2) * XS<T>::v, y0 - 2, j, &bars[s]);
    tma_load_3d(st + Ly::ZB, &emap, (x0 / 2 - 2) * XS<T>::v, y0 / 2 - 2, j, &bars[s]);
    tma_load_3d(st + Ly::ZB + Ly::EB, &bmap, (x0 - 2) * XS<T>::v, y0 - 1, j, &bars[s]);
    pend[s] = true;
  };
  int t = next_tile(blockIdx.x, G, total, tps, active);
  if (tid == 0 && t < total) issue(t, 0);
  int k = 0;
  for (; t < total; k++) {
    const int s = k & 1;
    const int tn = next_tile(t + G, G, total, tps, active);
    if (tid == 0 && tn < total) {
      fence_proxy_async_smem();
      issue(tn, s ^ 1);
    }
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k >> 1) & 1));
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(errflag, 2);
      break;
    }
    if (tid == 0) pend[s] = false;
    const int j = t / tps, tile = t - j * tps;
    const int y0 = (tile / tiles_x) * TY, x0 = (tile % tiles_x) * TX;
    C *Zs = reinterpret_cast<C *>(smem + s * Ly::STAGE);
    const C *Es = reinterpret_cast<const C *>(smem + s * Ly::STAGE + Ly::ZB);
    const C *Bs = reinterpret_cast<const C *>(smem + s * Ly::STAGE + Ly::ZB + Ly::EB);
    const Coef<T> cf = coef[j];
    const int ey0 = y0 / 2 - 2, ex0 = x0 / 2 - 2;
    // phase 1: z'' = z' + P e_c in place, rows y0-2.., cols x0-2.. (zero outside)
    for (int q = tid; q < ZH * ZW; q += kFT) {
      const int zr = q / ZW, zc = q - zr * ZW;
      const int i = y0 - 2 + zr, c = x0 - 2 + zc;
      C v = czero<C>();
      if ((unsigned)i < (unsigned)N && (unsigned)c < (unsigned)N) {
        auto E = [&](int I, int J) -> C { return Es[(I - ey0) * EW + (J - ex0)]; };
        C p;
        if (i & 1) {
          const int I = (i - 1) >> 1;
          if (c & 1) p = E(I, (c - 1) >> 1);
          else p = cscale(cadd(E(I, (c >> 1) - 1), E(I, c >> 1)), (T)0.5);
        } else {
          const int I1 = (i >> 1) - 1, I2 = i >> 1;
          if (c & 1) {
            const int J = (c - 1) >> 1;
            p = cscale(cadd(E(I1, J), E(I2, J)), (T)0.5);
          } else {
            const int J1 = (c >> 1) - 1, J2 = c >> 1;
            p = cscale(cadd(cadd(E(I1, J1), E(I1, J2)), cadd(E(I2, J1), E(I2, J2))), (T)0.25);
          }
        }
        v = cadd(Zs[q], p);
      }
      Zs[q] = v;
    }
    __syncthreads();
    // phase 2: rt of z'' on rows y0-1.., cols x0-1..
    for (int q = tid; q < RH * RW; q += kFT) {
      const int rr = q / RW, cc = q - rr * RW;
      const int i = y0 - 1 + rr, c = x0 - 1 + cc;
      C r = czero<C>();
      if ((unsigned)i < (unsigned)N && (unsigned)c < (unsigned)N) {
        const C *zc = &Zs[(rr + 1) * ZW + cc + 1];
        r = csub(cadd(Bs[rr * BW + cc + 1], cadd(cadd(zc[-ZW], zc[ZW]), cadd(zc[-1], zc[1]))),
                 cmul(cf.d, zc[0]));
      }
      R[q] = r;
    }
    __syncthreads();
    // phase 3: z''' = z'' + omega M rt on the tile
    for (int q = tid; q < TY * TX; q += kFT) {
      const int a = q / TX, b = q - a * TX;
      const int i = y0 + a, c = x0 + b;
      if (i < N && c < N) {
        const C *rc = &R[(a + 1) * RW + b + 1];
        C upd = cmul(cf.ca, rc[0]);
        const C e = cadd(cadd(rc[-RW], rc[RW]), cadd(rc[-1], rc[1]));
        const C kk = cadd(cadd(rc[-RW - 1], rc[-RW + 1]), cadd(rc[RW - 1], rc[RW + 1]));
        upd = cfma(cf.cb, e, upd);
        upd = cfma(cf.cc, kk, upd);
        stv<C>(zout, j, i, c, cadd(Zs[(a + 2) * ZW + b + 2], upd));
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    t = tn;
  }
  if (tid == 0)
    for (int s = 0; s < 2; s++)
      if (pend[s]) mbar_wait_bounded(&bars[s], (uint32_t)(((k + (s != (k & 1))) >> 1) & 1));
}

}  // namespace

template <typename T> FusedGeom fused_geom() {
  FusedGeom g;
  g.TX = FT<T>::TX;
  g.TY = FT<T>::TY;
  g.sr_zw = SRLayout<T>::ZW;
  g.sr_zh = SRLayout<T>::ZH;
  g.sr_bw = SRLayout<T>::BW;
  g.sr_bh = SRLayout<T>::BH;
  g.ps_zw = PSLayout<T>::ZW;
  g.ps_zh = PSLayout<T>::ZH;
  g.ps_ew = PSLayout<T>::EW;
  g.ps_eh = PSLayout<T>::EH;
  g.ps_bw = PSLayout<T>::BW;
  g.ps_bh = PSLayout<T>::BH;
  return g;
}

template <typename T> cudaError_t prepare_fused() {
  cudaError_t e;
  const int a = SRLayout<T>::SMEM, b = PSLayout<T>::SMEM;
#define PD_ATTR(K, S)                                                                     \
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, S);            \
  if (e != cudaSuccess) return e;
  PD_ATTR((k_smooth_restrict<T, false, false>), a)
  PD_ATTR((k_smooth_restrict<T, false, true>), a)
  PD_ATTR((k_smooth_restrict<T, true, false>), a)
  PD_ATTR((k_smooth_restrict<T, true, true>), a)
  PD_ATTR((k_prolong_smooth<T>), b)
#undef PD_ATTR
  return cudaSuccess;
}

template <typename T>
void launch_smooth_restrict(cudaStream_t s, int grid, const CUtensorMap &zmap,
                            const CUtensorMap &bmap, int N, int n, View zout, View bc,
                            const Coef<T> *coef, const int *active, bool z_zero, double *partials,
                            int part_stride, int *errflag) {
  const int smem = SRLayout<T>::SMEM;
  if (z_zero) {
    if (partials)
      k_smooth_restrict<T, true, true><<<grid, kFT, smem, s>>>(zmap, bmap, N, n, zout, bc, coef,
                                                               active, partials, part_stride, errflag);
    else
      k_smooth_restrict<T, true, false><<<grid, kFT, smem, s>>>(zmap, bmap, N, n, zout, bc, coef,
                                                                active, partials, part_stride, errflag);
  } else {
    if (partials)
      k_smooth_restrict<T, false, true><<<grid, kFT, smem, s>>>(zmap, bmap, N, n, zout, bc, coef,
                                                                active, partials, part_stride, errflag);
    else
      k_smooth_restrict<T, false, false><<<grid, kFT, smem, s>>>(zmap, bmap, N, n, zout, bc, coef,
                                                                 active, partials, part_stride, errflag);
  }
}

template <typename T>
void launch_prolong_smooth(cudaStream_t s, int grid, const CUtensorMap &zmap,
                           const CUtensorMap &emap, const CUtensorMap &bmap, int N, int n,
                           View zout, const Coef<T> *coef, const int *active, int *errflag) {
  k_prolong_smooth<T><<<grid, kFT, PSLayout<T>::SMEM, s>>>(zmap, emap, bmap, N, n, zout, coef,
                                                           active, errflag);
}

int fused_tiles(int N, int TX, int TY) { return ((N + TX - 1) / TX) * ((N + TY - 1) / TY); }

#define PD_INST_F(T)                                                                              \
  template FusedGeom fused_geom<T>();                                                             \
  template cudaError_t prepare_fused<T>();                                                        \
  template void launch_smooth_restrict<T>(cudaStream_t, int, const CUtensorMap &,                 \
                                          const CUtensorMap &, int, int, View, View,              \
                                          const Coef<T> *, const int *, bool, double *, int,      \
                                          int *);                                                 \
  template void launch_prolong_smooth<T>(cudaStream_t, int, const CUtensorMap &,                  \
                                         const CUtensorMap &, const CUtensorMap &, int, int, View, \
                                         const Coef<T> *, const int *, int *);

PD_INST_F(float)
PD_INST_F(double)

}  // namespace pd
