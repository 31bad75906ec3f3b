// Multigrid kernels for the n complex-shifted systems (A + lam_j I) z = b of eq. (2):
// the fused residual + additive Vanka smoother (Sec. 2, eq. (6)), residual + full
// weighting, linear interpolation, the per-shift convergence bookkeeping, and a
// kernel that runs whole cycles of the coarse levels inside one CTA per shift with
// the coarsest-grid direct solve (Sec. 3).
//
// All kernels work on the h^2-scaled residual rt = h^2 (b - L z):
//   rt = bt - (4 + eta) z + (z_N + z_S + z_W + z_E),  bt = h^2 b,  eta = lam h^2,
// so no 1/h^2 appears; the coarse right-hand side is bt_c = h_c^2 FW(r) = 4 FW(rt).
// Grid y (shift) of every launch runs over the n shifts; a CTA of an inactive
// (converged) shift returns at once.
#include "cplx.cuh"
#include "pd_internal.h"

namespace pd {

namespace {

template <typename C>
__device__ __forceinline__ C ldv(const View &v, int j, long long i, long long c) {
  return reinterpret_cast<const C *>(v.p)[j * v.plane + i * v.pitch + c];
}
template <typename C>
__device__ __forceinline__ void stv(const View &v, int j, long long i, long long c, C x) {
  reinterpret_cast<C *>(v.p)[j * v.plane + i * v.pitch + c] = x;
}

// Deterministic block sum of one double per thread; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < NT / 32; k++) s += red[k];
  return s;
}

constexpr int kSmTX = 32, kSmTY = 16, kSmThreads = 256;

// One smoothing step on a TY x TX tile: stage z with a halo of 2 and bt with a halo
// of 1, form rt on the tile plus a halo of 1 (zero outside the interior: the
// residual of boundary values is not part of M's sum), then apply the 9-point M.
// NORM: also write the tile's sum of |rt|^2 (the residual of z_in) to partials.
template <typename T, bool ZZERO, bool NORM, bool JAC>
__global__ void __launch_bounds__(kSmThreads)
k_smooth(int N, View zin, View zout, View b, T bscale, const Coef<T> *__restrict__ coef,
         const int *__restrict__ active, double *__restrict__ partials, int part_stride) {
  using C = typename Cx<T>::type;
  constexpr int TX = kSmTX, TY = kSmTY, ZW = TX + 4, ZH = TY + 4, RW = TX + 2, RH = TY + 2;
  __shared__ C sz[ZZERO ? 1 : ZH * ZW];
  __shared__ C sr[RH * RW];
  __shared__ double red[kSmThreads / 32];
  const int j = blockIdx.y;
  if (active && !active[j]) return;
  const int tiles_x = (N + TX - 1) / TX;
  const int tile = blockIdx.x;
  const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
  const int tid = threadIdx.x;
  const Coef<T> cf = coef[j];
  if (!ZZERO) {
    for (int t = tid; t < ZH * ZW; t += kSmThreads) {
      const int rr = t / ZW, cc = t - rr * ZW;
      const int gi = y0 - 2 + rr, gj = x0 - 2 + cc;
      C v = czero<C>();
      if ((unsigned)gi < (unsigned)N && (unsigned)gj < (unsigned)N) v = ldv<C>(zin, j, gi, gj);
      sz[t] = v;
    }
    __syncthreads();
  }
  for (int t = tid; t < RH * RW; t += kSmThreads) {
    const int rr = t / RW, cc = t - rr * RW;
    const int gi = y0 - 1 + rr, gj = x0 - 1 + cc;
    C r = czero<C>();
    if ((unsigned)gi < (unsigned)N && (unsigned)gj < (unsigned)N) {
      r = cscale(ldv<C>(b, j, gi, gj), bscale);
      if (!ZZERO) {
        const C *zc = &sz[(rr + 1) * ZW + cc + 1];
        const C nb = cadd(cadd(zc[-ZW], zc[ZW]), cadd(zc[-1], zc[1]));
        r = csub(cadd(r, nb), cmul(cf.d, zc[0]));
      }
    }
    sr[t] = r;
  }
  __syncthreads();
  T acc = 0;
  for (int t = tid; t < TY * TX; t += kSmThreads) {
    const int ty = t / TX, tx = t - ty * TX;
    const int gi = y0 + ty, gj = x0 + tx;
    if (gi < N && gj < N) {
      const C *rc = &sr[(ty + 1) * RW + tx + 1];
      const C rv = rc[0];
      C upd = cmul(cf.ca, rv);
      if (!JAC) {
        const C e = cadd(cadd(rc[-RW], rc[RW]), cadd(rc[-1], rc[1]));
        const C k = cadd(cadd(rc[-RW - 1], rc[-RW + 1]), cadd(rc[RW - 1], rc[RW + 1]));
        upd = cfma(cf.cb, e, upd);
        upd = cfma(cf.cc, k, upd);
      }
      const C zold = ZZERO ? czero<C>() : sz[(ty + 2) * ZW + tx + 2];
      stv<C>(zout, j, gi, gj, cadd(zold, upd));
      if (NORM) acc += rv.x * rv.x + rv.y * rv.y;
    }
  }
  if (NORM) {
    const double s = block_sum<kSmThreads>((double)acc, red);
    if (tid == 0) partials[(long long)j * part_stride + tile] = s;
  }
}

// Sum of |rt|^2 over a tile (used when there is no pre-smoothing step to carry it).
template <typename T, bool ZZERO>
__global__ void __launch_bounds__(kSmThreads)
k_resnorm(int N, View z, View b, T bscale, const Coef<T> *__restrict__ coef,
          const int *__restrict__ active, double *__restrict__ partials, int part_stride) {
  using C = typename Cx<T>::type;
  __shared__ double red[kSmThreads / 32];
  const int j = blockIdx.y;
  if (active && !active[j]) return;
  const int tiles_x = (N + kSmTX - 1) / kSmTX;
  const int tile = blockIdx.x;
  const int x0 = (tile % tiles_x) * kSmTX, y0 = (tile / tiles_x) * kSmTY;
  const Coef<T> cf = coef[j];
  double acc = 0.0;
  for (int t = threadIdx.x; t < kSmTX * kSmTY; t += kSmThreads) {
    const int gi = y0 + t / kSmTX, gj = x0 + t % kSmTX;
    if (gi < N && gj < N) {
      C r = cscale(ldv<C>(b, j, gi, gj), bscale);
      if (!ZZERO) {
        C nb = czero<C>();
        if (gi > 0) nb = cadd(nb, ldv<C>(z, j, gi - 1, gj));
        if (gi < N - 1) nb = cadd(nb, ldv<C>(z, j, gi + 1, gj));
        if (gj > 0) nb = cadd(nb, ldv<C>(z, j, gi, gj - 1));
        if (gj < N - 1) nb = cadd(nb, ldv<C>(z, j, gi, gj + 1));
        r = csub(cadd(r, nb), cmul(cf.d, ldv<C>(z, j, gi, gj)));
      }
      acc += cabs2(r);
    }
  }
  const double s = block_sum<kSmThreads>(acc, red);
  if (threadIdx.x == 0) partials[(long long)j * part_stride + tile] = s;
}

// Convergence test of Sec. 3 per shift (relative residual before each cycle), in a
// fixed summation order so that the stopping cycle is reproducible.
// stall > 0: also stop once a cycle reduced the relative residual by less than `stall`
// (the floor set by the rounding of z in the working precision has been reached).
// One warp per shift; the lanes' strided sums are combined in a fixed order.
__global__ void k_converge(int n, int ntiles, SolveState st, double tol, int maxit, double stall,
                           int cur_buf) {
  const int j = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= n || !st.active[j]) return;
  double s = 0.0;
  for (int t = lane; t < ntiles; t += 32) s += st.partials[(long long)j * st.max_tiles + t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  const int k = st.iters[j];
  if (k == 0) st.bn2[j] = s;
  const double bn2 = st.bn2[j];
  const double rr = bn2 > 0.0 ? sqrt(s / bn2) : 0.0;
  const double prev = st.relres[j];
  st.relres[j] = rr;
  if (st.hist && k < st.hist_stride) st.hist[(long long)j * st.hist_stride + k] = rr;
  const bool bad = !isfinite(s);
  if (bad) atomicOr(st.flags, 1);
  const bool stalled = stall > 0.0 && k >= 2 && rr > stall * prev;
  if (bad || rr <= tol || k >= maxit || stalled) {
    st.active[j] = 0;
    st.final_buf[j] = cur_buf;
    atomicSub(st.nactive, 1);
  } else {
    st.iters[j] = k + 1;
  }
}

// the convergence test of several instances in one launch: warp w of the launch tests the
// global shift w; task t owns the shifts j0 .. j0 + n - 1; batch_nactive counts down with
// every shift that stops
__global__ void k_converge_multi(const ConvTask *__restrict__ tasks, int ntasks, int total, double tol,
                                 int maxit, double stall, int cur_buf, int *batch_nactive) {
  const int g = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= total) return;
  int t = 0;
  while (t + 1 < ntasks && g >= tasks[t + 1].j0) t++;
  const ConvTask &k = tasks[t];
  const SolveState &st = k.st;
  const int j = g - k.j0;
  if (!st.active[j]) return;
  double s = 0.0;
  for (int q = lane; q < k.ntiles; q += 32) s += st.partials[(long long)j * st.max_tiles + q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  const int it = st.iters[j];
  if (it == 0) st.bn2[j] = s;
  const double bn2 = st.bn2[j];
  const double rr = bn2 > 0.0 ? sqrt(s / bn2) : 0.0;
  const double prev = st.relres[j];
  st.relres[j] = rr;
  if (st.hist && it < st.hist_stride) st.hist[(long long)j * st.hist_stride + it] = rr;
  const bool bad = !isfinite(s);
  if (bad) atomicOr(st.flags, 1);
  const bool stalled = stall > 0.0 && it >= 2 && rr > stall * prev;
  if (bad || rr <= tol || it >= maxit || stalled) {
    st.active[j] = 0;
    st.final_buf[j] = cur_buf;
    atomicSub(st.nactive, 1);
    atomicSub(batch_nactive, 1);
  } else {
    st.iters[j] = it + 1;
  }
}

// k_finalize for several instances (one thread per global shift)
__global__ void k_finalize_multi(const ConvTask *__restrict__ tasks, int ntasks, int total, int cur_buf,
                                 int *batch_nactive) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int t = 0;
  while (t + 1 < ntasks && g >= tasks[t + 1].j0) t++;
  const SolveState &st = tasks[t].st;
  const int j = g - tasks[t].j0;
  if (st.active[j]) {
    st.active[j] = 0;
    st.final_buf[j] = cur_buf;
    const int k = st.iters[j];
    if (st.hist && k < st.hist_stride) st.hist[(long long)j * st.hist_stride + k] = -1.0;
    atomicSub(st.nactive, 1);
    atomicSub(batch_nactive, 1);
  }
}

constexpr int kRsCT = 16;  // coarse points per tile side

// bt_c(I,J) = oscale * (1/4) sum_{di,dj} w rt(2I+1+di, 2J+1+dj), w = [1 2 1; 2 4 2; 1 2 1]
// (4 x full weighting of rt = h_c^2 FW(r) for oscale = 1).
template <typename T, bool ZZERO>
__global__ void __launch_bounds__(256)
k_residual_restrict(int Nf, View z, View b, T bscale, View bc, T oscale,
                    const Coef<T> *__restrict__ coef, const int *__restrict__ active) {
  using C = typename Cx<T>::type;
  constexpr int FR = 2 * kRsCT + 1, ZR = FR + 2;
  __shared__ C sz[ZZERO ? 1 : ZR * ZR];
  __shared__ C sr[FR * FR];
  const int j = blockIdx.y;
  if (active && !active[j]) return;
  const int Nc = (Nf - 1) / 2;
  const int tiles_x = (Nc + kRsCT - 1) / kRsCT;
  const int I0 = (blockIdx.x / tiles_x) * kRsCT, J0 = (blockIdx.x % tiles_x) * kRsCT;
  const int fi0 = 2 * I0, fj0 = 2 * J0;
  const Coef<T> cf = coef[j];
  if (!ZZERO) {
    for (int t = threadIdx.x; t < ZR * ZR; t += 256) {
      const int rr = t / ZR, cc = t - rr * ZR;
      const int gi = fi0 - 1 + rr, gj = fj0 - 1 + cc;
      C v = czero<C>();
      if ((unsigned)gi < (unsigned)Nf && (unsigned)gj < (unsigned)Nf) v = ldv<C>(z, j, gi, gj);
      sz[t] = v;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < FR * FR; t += 256) {
    const int rr = t / FR, cc = t - rr * FR;
    const int gi = fi0 + rr, gj = fj0 + cc;
    C r = czero<C>();
    if (gi < Nf && gj < Nf) {
      r = cscale(ldv<C>(b, j, gi, gj), bscale);
      if (!ZZERO) {
        const C *zc = &sz[(rr + 1) * ZR + cc + 1];
        const C nb = cadd(cadd(zc[-ZR], zc[ZR]), cadd(zc[-1], zc[1]));
        r = csub(cadd(r, nb), cmul(cf.d, zc[0]));
      }
    }
    sr[t] = r;
  }
  __syncthreads();
  const int ty = threadIdx.x / kRsCT, tx = threadIdx.x % kRsCT;
  const int I = I0 + ty, J = J0 + tx;
  if (I < Nc && J < Nc) {
    const C *rc = &sr[(2 * ty + 1) * FR + 2 * tx + 1];
    const C e = cadd(cadd(rc[-FR], rc[FR]), cadd(rc[-1], rc[1]));
    const C k = cadd(cadd(rc[-FR - 1], rc[-FR + 1]), cadd(rc[FR - 1], rc[FR + 1]));
    C s = cadd(cadd(cscale(rc[0], (T)4), cscale(e, (T)2)), k);
    stv<C>(bc, j, I, J, cscale(s, (T)0.25 * oscale));
  }
}

// z += P ec, P linear interpolation (= 4 FW^T): odd fine indices sit on coarse
// points, even ones halfway between (zero beyond the boundary).
template <typename T>
__global__ void __launch_bounds__(256)
k_prolong_add(int Nf, View z, View ec, const int *__restrict__ active) {
  using C = typename Cx<T>::type;
  const int j = blockIdx.z;
  if (active && !active[j]) return;
  const int i = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 32 + threadIdx.x;
  if (i >= Nf || c >= Nf) return;
  const int Nc = (Nf - 1) / 2;
  auto get = [&](int I, int J) -> C {
    return ((unsigned)I < (unsigned)Nc && (unsigned)J < (unsigned)Nc) ? ldv<C>(ec, j, I, J) : czero<C>();
  };
  C v;
  if (i & 1) {
    const int I = (i - 1) >> 1;
    if (c & 1) v = get(I, (c - 1) >> 1);
    else v = cscale(cadd(get(I, (c >> 1) - 1), get(I, c >> 1)), (T)0.5);
  } else {
    const int I1 = (i >> 1) - 1, I2 = i >> 1;
    if (c & 1) {
      const int J = (c - 1) >> 1;
      v = cscale(cadd(get(I1, J), get(I2, J)), (T)0.5);
    } else {
      const int J1 = (c >> 1) - 1, J2 = c >> 1;
      v = cscale(cadd(cadd(get(I1, J1), get(I1, J2)), cadd(get(I2, J1), get(I2, J2))), (T)0.25);
    }
  }
  stv<C>(z, j, i, c, cadd(ldv<C>(z, j, i, c), v));
}

// ---------------------------------------------------------------------------------
// Coarse levels inside one CTA per shift: z_l, bt_l, rt_l of levels start..L-1 live in
// shared memory; the cycle recursion (gamma, nu1, nu2) is the one of Sec. 3.  The
// recursion is unrolled at compile time over at most kMaxCoarseDepth levels, so the
// kernel needs no runtime call stack.
constexpr int kCoThreads = 512;

template <typename T>
__device__ void cta_residual(int N, const typename Cx<T>::type *z, const typename Cx<T>::type *b,
                             typename Cx<T>::type *r, typename Cx<T>::type d) {
  using C = typename Cx<T>::type;
  for (int p = threadIdx.x; p < N * N; p += kCoThreads) {
    const int i = p / N, c = p - i * N;
    C nb = czero<C>();
    if (i > 0) nb = cadd(nb, z[p - N]);
    if (i < N - 1) nb = cadd(nb, z[p + N]);
    if (c > 0) nb = cadd(nb, z[p - 1]);
    if (c < N - 1) nb = cadd(nb, z[p + 1]);
    r[p] = csub(cadd(b[p], nb), cmul(d, z[p]));
  }
}

template <typename T>
__device__ void cta_smooth(int N, typename Cx<T>::type *z, const typename Cx<T>::type *b,
                           typename Cx<T>::type *r, const Coef<T> &cf, bool jac) {
  using C = typename Cx<T>::type;
  cta_residual<T>(N, z, b, r, cf.d);
  __syncthreads();
  for (int p = threadIdx.x; p < N * N; p += kCoThreads) {
    const int i = p / N, c = p - i * N;
    C upd = cmul(cf.ca, r[p]);
    if (!jac) {
      auto R = [&](int di, int dc) -> C {
        const int ii = i + di, cc = c + dc;
        return ((unsigned)ii < (unsigned)N && (unsigned)cc < (unsigned)N) ? r[ii * N + cc] : czero<C>();
      };
      const C e = cadd(cadd(R(-1, 0), R(1, 0)), cadd(R(0, -1), R(0, 1)));
      const C k = cadd(cadd(R(-1, -1), R(-1, 1)), cadd(R(1, -1), R(1, 1)));
      upd = cfma(cf.cb, e, upd);
      upd = cfma(cf.cc, k, upd);
    }
    z[p] = cadd(z[p], upd);
  }
  __syncthreads();
}



// shared-memory base and per-level element offsets of z_l (bt_l = z_l + N_l^2,
// rt_l = z_l + 2 N_l^2)
template <typename T> struct CtaMem {
  typename Cx<T>::type *base;
  const int *off;
  __device__ typename Cx<T>::type *z(int l, int N) const { return base + off[l]; }
  __device__ typename Cx<T>::type *b(int l, int N) const { return base + off[l] + N * N; }
  __device__ typename Cx<T>::type *r(int l, int N) const { return base + off[l] + 2 * N * N; }
};

template <typename T, int D>
__device__ __forceinline__ void cta_cycle(int l, const CoarseArgs<T> &a, const CtaMem<T> &g) {
  using C = typename Cx<T>::type;
  const int j = blockIdx.x - a.block0;
  const int N = a.plan.Ns[l];
  if (l == a.plan.L - 1) {
    const int m = N * N;
    const C *inv = a.cinv + (long long)j * m * m;
    const C *bl = g.b(l, N);
    C *zl = g.z(l, N);
    for (int p = threadIdx.x; p < m; p += kCoThreads) {
      C s = czero<C>();
      for (int q = 0; q < m; q++) s = cfma(inv[(long long)p * m + q], bl[q], s);
      zl[p] = s;
    }
    __syncthreads();
    return;
  }
  if constexpr (D > 0) {
    const Coef<T> cf = a.coef[(long long)l * a.n + j];
    C *z = g.z(l, N), *b = g.b(l, N), *r = g.r(l, N);
    for (int s = 0; s < a.plan.nu1; s++) cta_smooth<T>(N, z, b, r, cf, a.plan.jacobi);
    cta_residual<T>(N, z, b, r, cf.d);
    __syncthreads();
    const int Nc = (N - 1) / 2;
    C *bc = g.b(l + 1, Nc), *zc = g.z(l + 1, Nc);
    for (int p = threadIdx.x; p < Nc * Nc; p += kCoThreads) {
      const int I = p / Nc, J = p - I * Nc;
      const C *rc = r + (2 * I + 1) * N + 2 * J + 1;
      const C e = cadd(cadd(rc[-N], rc[N]), cadd(rc[-1], rc[1]));
      const C k = cadd(cadd(rc[-N - 1], rc[-N + 1]), cadd(rc[N - 1], rc[N + 1]));
      bc[p] = cscale(cadd(cadd(cscale(rc[0], (T)4), cscale(e, (T)2)), k), (T)0.25);
      zc[p] = czero<C>();
    }
    __syncthreads();
    for (int gm = 0; gm < a.plan.gamma; gm++) cta_cycle<T, D - 1>(l + 1, a, g);
    for (int p = threadIdx.x; p < N * N; p += kCoThreads) {
      const int i = p / N, c = p - i * N;
      auto get = [&](int I, int J) -> C {
        return ((unsigned)I < (unsigned)Nc && (unsigned)J < (unsigned)Nc) ? zc[I * Nc + J] : czero<C>();
      };
      C v;
      if (i & 1) {
        const int I = (i - 1) >> 1;
        if (c & 1) v = get(I, (c - 1) >> 1);
        else v = cscale(cadd(get(I, (c >> 1) - 1), get(I, c >> 1)), (T)0.5);
      } else {
        const int I1 = (i >> 1) - 1, I2 = i >> 1;
        if (c & 1) {
          const int J = (c - 1) >> 1;
          v = cscale(cadd(get(I1, J), get(I2, J)), (T)0.5);
        } else {
          const int J1 = (c >> 1) - 1, J2 = c >> 1;
          v = cscale(cadd(cadd(get(I1, J1), get(I1, J2)), cadd(get(I2, J1), get(I2, J2))), (T)0.25);
        }
      }
      z[p] = cadd(z[p], v);
    }
    __syncthreads();
    for (int s = 0; s < a.plan.nu2; s++) cta_smooth<T>(N, z, b, r, cf, a.plan.jacobi);
  }
}

// mode 0: ncycles cycles at level `start` from z = 0 (or from zio when load_z);
// mode 1: the whole solve of eq. (2) at level start = 0 with the relative-residual
// test of Sec. 3 before each cycle; writes iters/relres/final_buf of the state.
template <typename T>
__device__ __forceinline__ void coarse_run(const CoarseArgs<T> &a, View b, T bscale, View zio,
                                           const int *__restrict__ active, int ncycles, int load_z,
                                           int solve_mode, double tol, int maxit, SolveState st) {
  using C = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kCoThreads / 32];
  __shared__ int off[kMaxLevels];
  __shared__ int stop;
  const int j = blockIdx.x - a.block0;
  if (active && !active[j]) return;
  if (threadIdx.x == 0) {
    int o = 0;
    for (int l = a.start; l < a.plan.L; l++) {
      off[l] = o;
      o += 3 * a.plan.Ns[l] * a.plan.Ns[l];
    }
  }
  __syncthreads();
  const CtaMem<T> g{reinterpret_cast<C *>(smem_raw), off};
  const int l0 = a.start, N = a.plan.Ns[l0];
  C *z0 = g.z(l0, N), *b0 = g.b(l0, N), *r0 = g.r(l0, N);
  for (int q = threadIdx.x; q < N * N; q += kCoThreads) {
    const int i = q / N, c = q - i * N;
    b0[q] = cscale(ldv<C>(b, j, i, c), bscale);
    z0[q] = load_z ? ldv<C>(zio, j, i, c) : czero<C>();
  }
  __syncthreads();
  if (!solve_mode) {
    for (int k = 0; k < ncycles; k++) cta_cycle<T, kMaxCoarseDepth>(l0, a, g);
  } else {
    const Coef<T> cf = a.coef[(long long)l0 * a.n + j];
    double bn2 = 0.0, rr = 0.0;
    int k = 0;
    for (;;) {
      cta_residual<T>(N, z0, b0, r0, cf.d);
      __syncthreads();
      double acc = 0.0;
      for (int q = threadIdx.x; q < N * N; q += kCoThreads) acc += cabs2(r0[q]);
      const double s = block_sum<kCoThreads>(acc, red);
      if (threadIdx.x == 0) {
        if (k == 0) bn2 = s;
        rr = bn2 > 0.0 ? sqrt(s / bn2) : 0.0;
        if (st.hist && k < st.hist_stride) st.hist[(long long)j * st.hist_stride + k] = rr;
        const bool bad = !isfinite(s);
        if (bad) atomicOr(st.flags, 1);
        stop = (bad || rr <= tol || k >= maxit);
      }
      __syncthreads();
      if (stop) break;
      cta_cycle<T, kMaxCoarseDepth>(l0, a, g);
      k++;
    }
    if (threadIdx.x == 0) {
      st.iters[j] = k;
      st.relres[j] = rr;
      st.bn2[j] = bn2;
      st.final_buf[j] = 0;
      st.active[j] = 0;
      atomicSub(st.nactive, 1);
    }
  }
  for (int q = threadIdx.x; q < N * N; q += kCoThreads) {
    const int i = q / N, c = q - i * N;
    stv<C>(zio, j, i, c, z0[q]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kCoThreads)
k_coarse(CoarseArgs<T> a, View b, T bscale, View zio, const int *__restrict__ active, int ncycles,
         int load_z, int solve_mode, double tol, int maxit, SolveState st) {
  coarse_run<T>(a, b, bscale, zio, active, ncycles, load_z, solve_mode, tol, maxit, st);
}

// the coarse levels of several instances in one launch (mode 0, from z = 0): task t owns
// the CTAs block0 .. block0 + n - 1 of its arguments
template <typename T>
__global__ void __launch_bounds__(kCoThreads)
k_coarse_multi(const CoarseTask<T> *__restrict__ tasks, int ntasks, int ncycles) {
  int t = 0;
  while (t + 1 < ntasks && (int)blockIdx.x >= tasks[t + 1].a.block0) t++;
  const CoarseTask<T> &k = tasks[t];
  coarse_run<T>(k.a, k.b, (T)1, k.z, k.active, ncycles, 0, 0, 0.0, 0, SolveState{});
}

template <typename T>
__global__ void k_copy_scale(int N, View dst, View src, T scale) {
  using C = typename Cx<T>::type;
  const int j = blockIdx.z;
  const int i = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 32 + threadIdx.x;
  if (i >= N || c >= N) return;
  stv<C>(dst, j, i, c, cscale(ldv<C>(src, j, i, c), scale));
}

template <typename T>
__global__ void k_gather_final(int N, View dst, View z0, View z1, const int *__restrict__ final_buf) {
  using C = typename Cx<T>::type;
  const int j = blockIdx.z;
  const int i = blockIdx.y * 8 + threadIdx.y, c = blockIdx.x * 32 + threadIdx.x;
  if (i >= N || c >= N) return;
  const View &src = (final_buf && final_buf[j]) ? z1 : z0;
  stv<C>(dst, j, i, c, ldv<C>(src, j, i, c));
}

__global__ void k_reset_state(int n, SolveState st) {
  const int j = threadIdx.x;
  if (j < n) {
    st.active[j] = 1;
    st.iters[j] = 0;
    st.final_buf[j] = 0;
    st.bn2[j] = 0.0;
    st.relres[j] = 0.0;
  }
  if (j == 0) {
    *st.nactive = n;
    *st.flags = 0;
  }
}

// Ends a solve after its last permitted cycle without another residual: every shift
// still iterating keeps the iterate in buffer cur_buf and its last relative residual.
__global__ void k_finalize(int n, SolveState st, int cur_buf) {
  const int j = threadIdx.x;
  if (j < n && st.active[j]) {
    st.active[j] = 0;
    st.final_buf[j] = cur_buf;
    const int k = st.iters[j];
    if (st.hist && k < st.hist_stride) st.hist[(long long)j * st.hist_stride + k] = -1.0;
    atomicSub(st.nactive, 1);
  }
}

}  // namespace

void launch_reset_state(cudaStream_t s, int n, SolveState st) { k_reset_state<<<1, 128, 0, s>>>(n, st); }
void launch_finalize(cudaStream_t s, int n, SolveState st, int cur_buf) {
  k_finalize<<<1, 128, 0, s>>>(n, st, cur_buf);
}

int smooth_tiles(int N) { return ((N + kSmTX - 1) / kSmTX) * ((N + kSmTY - 1) / kSmTY); }

template <typename T>
void launch_smooth(cudaStream_t s, int N, int n, View zin, View zout, View b, T bscale,
                   const Coef<T> *coef, const int *active, bool z_zero, bool jacobi,
                   double *partials, int part_stride) {
  dim3 grid(smooth_tiles(N), n);
  const bool norm = partials != nullptr;
#define PD_SM(ZZ, NM, JC)                                                                      \
  k_smooth<T, ZZ, NM, JC><<<grid, kSmThreads, 0, s>>>(N, zin, zout, b, bscale, coef, active, \
                                                       partials, part_stride)
  if (z_zero) {
    if (norm) { if (jacobi) PD_SM(true, true, true); else PD_SM(true, true, false); }
    else { if (jacobi) PD_SM(true, false, true); else PD_SM(true, false, false); }
  } else {
    if (norm) { if (jacobi) PD_SM(false, true, true); else PD_SM(false, true, false); }
    else { if (jacobi) PD_SM(false, false, true); else PD_SM(false, false, false); }
  }
#undef PD_SM
}

template <typename T>
void launch_resnorm(cudaStream_t s, int N, int n, View z, View b, T bscale, const Coef<T> *coef,
                    const int *active, bool z_zero, double *partials, int part_stride) {
  dim3 grid(smooth_tiles(N), n);
  if (z_zero)
    k_resnorm<T, true><<<grid, kSmThreads, 0, s>>>(N, z, b, bscale, coef, active, partials, part_stride);
  else
    k_resnorm<T, false><<<grid, kSmThreads, 0, s>>>(N, z, b, bscale, coef, active, partials, part_stride);
}

void launch_converge(cudaStream_t s, int n, int ntiles, SolveState st, double tol, int maxit,
                     double stall, int cur_buf) {
  k_converge<<<(n + 3) / 4, 128, 0, s>>>(n, ntiles, st, tol, maxit, stall, cur_buf);
}

template <typename T>
void launch_residual_restrict(cudaStream_t s, int Nf, int n, View z, View b, T bscale, View bc,
                              T oscale, const Coef<T> *coef, const int *active, bool z_zero) {
  const int Nc = (Nf - 1) / 2;
  const int t = (Nc + kRsCT - 1) / kRsCT;
  dim3 grid(t * t, n);
  if (z_zero)
    k_residual_restrict<T, true><<<grid, 256, 0, s>>>(Nf, z, b, bscale, bc, oscale, coef, active);
  else
    k_residual_restrict<T, false><<<grid, 256, 0, s>>>(Nf, z, b, bscale, bc, oscale, coef, active);
}

template <typename T>
void launch_prolong_add(cudaStream_t s, int Nf, int n, View z, View ec, const int *active) {
  dim3 grid((Nf + 31) / 32, (Nf + 7) / 8, n);
  k_prolong_add<T><<<grid, dim3(32, 8), 0, s>>>(Nf, z, ec, active);
}

template <typename T>
size_t coarse_smem_bytes(const CoarsePlan &plan, int start) {
  size_t e = 0;
  for (int l = start; l < plan.L; l++) e += 3ull * plan.Ns[l] * plan.Ns[l];
  return e * sizeof(typename Cx<T>::type);
}

template <typename T>
cudaError_t prepare_coarse(size_t smem) {
  const cudaError_t e = cudaFuncSetAttribute(k_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_coarse_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
void launch_coarse(cudaStream_t s, const CoarsePlan &plan, int start, int n, View b, T bscale,
                   View z, const Coef<T> *coef, const typename Cx<T>::type *cinv,
                   const int *active, int ncycles, int load_z, int solve_mode, double tol,
                   int maxit, SolveState st) {
  CoarseArgs<T> a;
  a.plan = plan;
  a.n = n;
  a.start = start;
  a.block0 = 0;
  a.coef = coef;
  a.cinv = cinv;
  const size_t smem = coarse_smem_bytes<T>(plan, start);
  k_coarse<T><<<n, kCoThreads, smem, s>>>(a, b, bscale, z, active, ncycles, load_z, solve_mode,
                                          tol, maxit, st);
}

template <typename T>
void launch_coarse_multi(cudaStream_t s, const CoarseTask<T> *tasks, int ntasks, int blocks, size_t smem,
                         int ncycles) {
  k_coarse_multi<T><<<blocks, kCoThreads, smem, s>>>(tasks, ntasks, ncycles);
}

void launch_converge_multi(cudaStream_t s, const ConvTask *tasks, int ntasks, int total, double tol,
                           int maxit, double stall, int cur_buf, int *batch_nactive) {
  k_converge_multi<<<(total + 3) / 4, 128, 0, s>>>(tasks, ntasks, total, tol, maxit, stall, cur_buf,
                                                   batch_nactive);
}

void launch_finalize_multi(cudaStream_t s, const ConvTask *tasks, int ntasks, int total, int cur_buf,
                           int *batch_nactive) {
  k_finalize_multi<<<(total + 127) / 128, 128, 0, s>>>(tasks, ntasks, total, cur_buf, batch_nactive);
}

template <typename T>
void launch_copy_scale(cudaStream_t s, int N, int n, View dst, View src, T scale) {
  dim3 grid((N + 31) / 32, (N + 7) / 8, n);
  k_copy_scale<T><<<grid, dim3(32, 8), 0, s>>>(N, dst, src, scale);
}

template <typename T>
void launch_gather_final(cudaStream_t s, int N, int n, View dst, View z0, View z1,
                         const int *final_buf) {
  dim3 grid((N + 31) / 32, (N + 7) / 8, n);
  k_gather_final<T><<<grid, dim3(32, 8), 0, s>>>(N, dst, z0, z1, final_buf);
}

#define PD_INST(T)                                                                                  \
  template void launch_smooth<T>(cudaStream_t, int, int, View, View, View, T, const Coef<T> *,     \
                                 const int *, bool, bool, double *, int);                          \
  template void launch_resnorm<T>(cudaStream_t, int, int, View, View, T, const Coef<T> *,          \
                                  const int *, bool, double *, int);                               \
  template void launch_residual_restrict<T>(cudaStream_t, int, int, View, View, T, View, T,        \
                                            const Coef<T> *, const int *, bool);                   \
  template void launch_prolong_add<T>(cudaStream_t, int, int, View, View, const int *);            \
  template size_t coarse_smem_bytes<T>(const CoarsePlan &, int);                                   \
  template cudaError_t prepare_coarse<T>(size_t);                                                  \
  template void launch_coarse<T>(cudaStream_t, const CoarsePlan &, int, int, View, T, View,        \
                                 const Coef<T> *, const typename Cx<T>::type *, const int *, int,  \
                                 int, int, double, int, SolveState);                               \
  template void launch_coarse_multi<T>(cudaStream_t, const CoarseTask<T> *, int, int, size_t, int); \
  template void launch_copy_scale<T>(cudaStream_t, int, int, View, View, T);                       \
  template void launch_gather_final<T>(cudaStream_t, int, int, View, View, View, const int *);

PD_INST(double)
PD_INST(float)

}  // namespace pd
