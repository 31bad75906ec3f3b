// C ABI of libparadiag.so: context setup and the orchestration of the ParaDIAG step
// (Sec. 1, eq. (1)-(2)) around the multigrid of Sec. 2-3.  Every arithmetic step of
// a solve runs in the kernels of mg_kernels.cu and transforms.cu; this file only
// allocates, launches and reads back convergence information.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "pd_internal.h"

using namespace pd;

namespace {

constexpr size_t kCoarseSmemLimit = 200 * 1024;

struct LevelBufs {
  int N = 0;
  long long P = 0;        // row pitch (elements) of the internal arrays
  void *z[2] = {nullptr, nullptr};
  void *b = nullptr;
  // TMA maps of the fused kernels (boxes with halos, zero fill outside the grid)
  CUtensorMap sr_z[2], sr_b;          // smooth+restrict: z and bt of this level
  CUtensorMap ps_z[2], ps_e[2], ps_b; // prolong+smooth: z of this level, z of the next, bt
  bool maps = false;
  int variant = 2;  // fused implementation of this level: 1 TMA tiles, 2 warp streams
  int seg = 128;    // rows per warp-stream segment
};

template <typename T> struct Prec {
  using C = typename Cx<T>::type;
  std::vector<LevelBufs> lv;
  Coef<T> *coef = nullptr;  // [L][n]
  C *cinv = nullptr;        // [n][mc*mc]
  C *Wf = nullptr;          // V^{-1}, n x n
  C *Wi = nullptr;          // V, n x n
  // TF32 split operands of the tensor-core transforms (forward scaled by h^2 and unscaled)
  float *tc_fwd_hi = nullptr, *tc_fwd_lo = nullptr, *tc_inv_hi = nullptr, *tc_inv_lo = nullptr;
  int tc_grid_fwd = 0, tc_grid_inv = 0;  // CTAs of the tensor-core transform launches
  float *tc_fwd1_hi = nullptr, *tc_fwd1_lo = nullptr;
  bool tc = false;
  // FFT route for an alpha-circulant V: weights alpha^{k/n} h^2/(kappa n), alpha^{k/n}/n
  // (unscaled) and alpha^{-k/n}; twiddles e^{+-2 pi i t/n}
  T *fft_wf = nullptr, *fft_wf1 = nullptr, *fft_wi = nullptr;
  C *fft_twf = nullptr, *fft_twi = nullptr;
  bool fft = false;
};

}  // namespace

struct pd_ctx {
  int N = 0, n = 0, L = 0, lc = 0;
  pd_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<double> shifts, omega, V, Vinv, B, u0coef;
  bool have_V = false, have_B = false;
  std::vector<int> Ns;
  CoarsePlan plan{};
  Prec<double> p64;
  Prec<float> p32;
  int cur[kMaxLevels] = {0};
  SolveState st{};
  void *state_mem = nullptr;
  int *h_pinned = nullptr;     // [2] nactive slots, [2..] flags
  int *h_iters = nullptr;      // pinned [n]
  double *h_relres = nullptr;  // pinned [n]
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double *d_u0coef = nullptr;
  int *d_Bptr = nullptr, *d_Bcol = nullptr;
  double *d_Bval = nullptr;
  double *d_r = nullptr;       // refinement residual [n][N][N] (general B)
  float *d_r32 = nullptr;      // refinement residual in FP32 (bidiagonal B)
  float2 *d_fcache = nullptr;  // fhat in float-float, written by a solve's first residual
  bool bidiag = false;         // B has nonzeros only at (k,k) and (k,k+boff mod n)
  int boff = -1;
  double *d_bd = nullptr, *d_bs = nullptr;
  float4 *d_kbd = nullptr;     // (bd_k, bs_k) as float-float pairs (FP64-free residual)
  float2 *d_ku0 = nullptr;     // u0coef_k as float-float pairs
  float2 ihf{0.f, 0.f};        // kappa / h^2 as a float-float pair
  int fsig = 0;                // scale exponent of the ||fhat|| sums (kept between solves)
  double fnorm = -1.0;         // ||fhat|| of the running refinement
  std::vector<double> outer_hist;  // relative residual of eq. (1) after each step of the
                                   // last paradiag_solve
  double *d_part = nullptr;    // all-at-once residual partial sums
  double *h_part = nullptr;    // pinned copy
  unsigned long long *d_imag = nullptr;
  double *d_stage_f = nullptr, *d_stage_u = nullptr, *d_stage_u0 = nullptr;
  // pipelined host solves: copy streams (host-to-device, device-to-host: the host link
  // carries both directions at once) and two staging sets (f, u, u0)
  cudaStream_t copy_stream = nullptr, copy_stream_out = nullptr;
  double *d_pf[2] = {nullptr, nullptr}, *d_pu[2] = {nullptr, nullptr}, *d_pu0[2] = {nullptr, nullptr};
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  long long launches = 0;
  int num_sms = 0;
  double kappa = 1.0;     // A is scaled by kappa in eq. (1); the multigrid sees lam / kappa
  int stream_grid = 0;    // persistent grid of the streaming kernels
  // instrumentation: event pairs around launches, resolved after each solve
  bool prof_on = false;
  int cur_cyc = -1;                 // cycle of the running batched solve, -1 outside
  double stall = 0.0;               // stall ratio of the running solve (0: off)
  int *h_hist = nullptr;            // pinned [maxit + 2]: active shifts after each cycle's test
  std::vector<cudaEvent_t> prof_ev; // 2 per pair
  std::vector<int> prof_free;
  struct ProfRec {
    int kc, idx, cyc, phase;
    double bytes_per_shift;
  };
  std::vector<ProfRec> prof_pending;
  double prof_ms[PD_KC_COUNT] = {0}, prof_bytes[PD_KC_COUNT] = {0};
  long long prof_n[PD_KC_COUNT] = {0};
  // FP64 refinement of the shifted systems (shifted_solve_refined, batches)
  int *d_frozen = nullptr, *h_frozen = nullptr;  // [n] shift done: zero RHS, no update
  double2 *d_c1 = nullptr;                       // [n] lam_j + 4 kappa / h^2
  double2 *d_lam = nullptr;                      // [n] lam_j
  double *d_srpart = nullptr, *h_srpart = nullptr;  // [2][n][blocks] residual partial sums
  float *d_rsc = nullptr, *h_rsc = nullptr;  // [n] power-of-two scale of each shift's FP32 RHS
  // CUDA graphs of whole cycles, keyed by everything a cycle's launches depend on
  struct CycleGraph {
    int prec, zzero, cur0, cmax;
    double tol, stall;
    cudaGraphExec_t exec;
    int cur_after[kMaxLevels];
    long long launches;
  };
  std::vector<CycleGraph> graphs;
  bool graphs_ok = true;  // cleared when a capture fails: launches go one by one
  std::string err;
  std::vector<void *> allocs;
};

namespace {

struct CudaFail {
  cudaError_t e;
};

void ck(pd_ctx *c, cudaError_t e) {
  if (e != cudaSuccess) {
    if (c) c->err = cudaGetErrorString(e);
    throw CudaFail{e};
  }
}

void ck_launch(pd_ctx *c, int count = 1) {
  c->launches += count;
  ck(c, cudaGetLastError());
}

// phase of a launch for byte accounting: 0 all n shifts, 1 the shifts active when the
// cycle started (before its convergence test), 2 those active after it
int prof_begin(pd_ctx *c) {
  if (!c->prof_on) return -1;
  if (c->prof_free.empty()) {
    const int idx = (int)c->prof_ev.size() / 2;
    cudaEvent_t a, b;
    ck(c, cudaEventCreate(&a));
    ck(c, cudaEventCreate(&b));
    c->prof_ev.push_back(a);
    c->prof_ev.push_back(b);
    c->prof_free.push_back(idx);
  }
  const int idx = c->prof_free.back();
  c->prof_free.pop_back();
  ck(c, cudaEventRecord(c->prof_ev[2 * idx], c->stream));
  return idx;
}

void prof_end(pd_ctx *c, int idx, int kc, double bytes_per_shift, int phase) {
  if (idx < 0) return;
  ck(c, cudaEventRecord(c->prof_ev[2 * idx + 1], c->stream));
  if (c->cur_cyc < 0) phase = 0;
  c->prof_pending.push_back({kc, idx, c->cur_cyc, phase, bytes_per_shift});
}

// after a stream synchronisation: turn pending event pairs into totals
void prof_resolve(pd_ctx *c) {
  for (const auto &r : c->prof_pending) {
    float ms = 0.f;
    ck(c, cudaEventElapsedTime(&ms, c->prof_ev[2 * r.idx], c->prof_ev[2 * r.idx + 1]));
    double cnt = c->n;
    if (r.phase == 1) cnt = r.cyc == 0 ? c->n : c->h_hist[r.cyc - 1];
    if (r.phase == 2) cnt = c->h_hist[r.cyc];
    c->prof_ms[r.kc] += ms;
    c->prof_n[r.kc] += 1;
    c->prof_bytes[r.kc] += cnt * r.bytes_per_shift;
    c->prof_free.push_back(r.idx);
  }
  c->prof_pending.clear();
}

#define PD_PROF(kc, bytes, phase, ...)          \
  do {                                         \
    const int pi_ = prof_begin(c);             \
    __VA_ARGS__;                               \
    prof_end(c, pi_, (kc), (bytes), (phase));  \
  } while (0)

template <typename P> P dalloc(pd_ctx *c, size_t bytes) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    throw std::bad_alloc();
  }
  c->allocs.push_back(p);
  return reinterpret_cast<P>(p);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder(pd_ctx *c) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    ck(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) {
      c->err = "cuTensorMapEncodeTiled unavailable";
      throw CudaFail{cudaErrorNotSupported};
    }
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3D map of a [n][N][P] array of complex values (e 8-byte words each) with a box of
// bw x bh complex elements of one shift; reads outside [0,N)^2 return zeros
CUtensorMap grid_map(pd_ctx *c, void *base, int N, long long P, int n, int e, int bw, int bh) {
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)N * e, (cuuint64_t)N, (cuuint64_t)n};
  cuuint64_t strides[2] = {(cuuint64_t)P * 8 * e, (cuuint64_t)N * P * 8 * e};
  cuuint32_t box[3] = {(cuuint32_t)(bw * e), (cuuint32_t)bh, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = tensor_map_encoder(c)(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides,
                                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                           CU_TENSOR_MAP_SWIZZLE_NONE,
                                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    c->err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    throw CudaFail{cudaErrorInvalidValue};
  }
  return m;
}

View view(void *p, int N, long long P) { return View{p, P, (long long)N * P}; }
View uview(const void *p, int N) { return View{const_cast<void *>(p), N, (long long)N * N}; }

template <typename T> Prec<T> &prec(pd_ctx *c);
template <> Prec<double> &prec<double>(pd_ctx *c) { return c->p64; }
template <> Prec<float> &prec<float>(pd_ctx *c) { return c->p32; }

double hl(const pd_ctx *c, int l) { return 1.0 / (c->Ns[l] + 1); }
// scale of a right-hand side of level l in the kernels' form: h_l^2 / kappa
double rs(const pd_ctx *c, int l) { return hl(c, l) * hl(c, l) / c->kappa; }

// partial sums of the all-at-once residual kernels (the larger of the two grids)
int part_blocks(const pd_ctx *c) { return std::max(allatonce_blocks(), residual_fx_blocks(c->num_sms)); }

// Set-up autotuner of the fused kernels: on each global-memory level, times the
// smoothing+restriction and interpolation+smoothing pair of every candidate (warp streams
// with 4, 8, 16, 32, 64, 128 or 256 rows per segment) on the context's own (zeroed) buffers,
// all shifts active, and keeps the fastest.  The TMA tiles are a candidate only when
// cfg.fused_variant = 1 asks for them: timed beside the warp streams they lost on every
// level of grids 127..2047 (pd_fused_choice records the choices).
template <typename T>
void autotune_fused(pd_ctx *c) {
  Prec<T> &P = prec<T>(c);
  const int n = c->n;
  const FusedGeom g = fused_geom<T>();
  const int segs[7] = {4, 8, 16, 32, 64, 128, 256};
  cudaEvent_t e0, e1;
  ck(c, cudaEventCreate(&e0));
  ck(c, cudaEventCreate(&e1));
  int *dummy_err = c->st.flags;
  for (int l = 0; l < c->L - 1; l++) {
    LevelBufs &B = P.lv[l], &Bc = P.lv[l + 1];
    if (!B.maps) continue;
    const size_t bytes = (size_t)n * B.N * B.P * sizeof(typename Cx<T>::type);
    const size_t bytesc = (size_t)n * Bc.N * Bc.P * sizeof(typename Cx<T>::type);
    for (int q = 0; q < 2; q++) {
      ck(c, cudaMemsetAsync(B.z[q], 0, bytes, c->stream));
      ck(c, cudaMemsetAsync(Bc.z[q], 0, bytesc, c->stream));
    }
    ck(c, cudaMemsetAsync(B.b, 0, bytes, c->stream));
    const View b = view(B.b, B.N, B.P), z0 = view(B.z[0], B.N, B.P), z1 = view(B.z[1], B.N, B.P);
    const View bc = view(Bc.b, Bc.N, Bc.P), ec = view(Bc.z[0], Bc.N, Bc.P);
    const Coef<T> *cf = P.coef + (size_t)l * n;
    const int grid = std::max(1, std::min(c->num_sms, n * fused_tiles(B.N, g.TX, g.TY)));
    float best = 1e30f;
    int bv = 2, bs = 128;
    for (int cand = 0; cand < 8; cand++) {
      const int variant = cand == 0 ? 1 : 2, seg = cand == 0 ? 0 : segs[cand - 1];
      if ((c->cfg.fused_variant == 0 ? 2 : c->cfg.fused_variant) != variant) continue;
      if (variant == 2 && seg > 2 * B.N) continue;
      float tmin = 1e30f;
      for (int rep = 0; rep < 3; rep++) {
        ck(c, cudaEventRecord(e0, c->stream));
        if (variant == 1) {
          launch_smooth_restrict<T>(c->stream, grid, B.sr_z[0], B.sr_b, B.N, n, z1, bc, cf, nullptr,
                                    false, nullptr, 0, dummy_err);
          launch_prolong_smooth<T>(c->stream, grid, B.ps_z[1], B.ps_e[0], B.ps_b, B.N, n, z0, cf,
                                   nullptr, dummy_err);
        } else {
          launch_sr_stream<T>(c->stream, c->stream_grid, B.N, n, seg, z0, b, z1, bc, cf, nullptr,
                              false, nullptr, 0);
          launch_ps_stream<T>(c->stream, c->stream_grid, B.N, n, seg, z1, ec, b, z0, cf, nullptr);
        }
        ck(c, cudaEventRecord(e1, c->stream));
        ck(c, cudaEventSynchronize(e1));
        ck(c, cudaGetLastError());
        float ms = 0.f;
        ck(c, cudaEventElapsedTime(&ms, e0, e1));
        tmin = std::min(tmin, ms);
      }
      c->launches += 6;
      if (tmin < best) {
        best = tmin;
        bv = variant;
        bs = seg;
      }
    }
    B.variant = bv;
    B.seg = bs > 0 ? bs : 128;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// True when the context's V and V^{-1} are those of the alpha-circulant backward-Euler B
// (pd_alpha_circulant) for some alpha in (0, 1], to 1e-12 relative: the FFT route applies.
bool alpha_circulant_alpha(const pd_ctx *c, double *alpha_out) {
  const int n = c->n;
  if (n < 2) return false;
  const double v10 = c->V[2 * (size_t)n];  // V[1][0] = alpha^{-1/n}
  if (!(v10 >= 1.0) || c->V[2 * (size_t)n + 1] != 0.0) return false;
  const double alpha = std::pow(v10, -(double)n);
  if (!(alpha > 0.0 && alpha <= 1.0)) return false;
  double vmax = 0.0, imax = 0.0, dv = 0.0, di = 0.0;
  for (int k = 0; k < n; k++)
    for (int j = 0; j < n; j++) {
      const size_t e = (size_t)k * n + j;
      const double ang = 2.0 * M_PI * (double)((long long)k * j % n) / n;
      const std::complex<double> v = std::pow(alpha, -(double)k / n) * std::polar(1.0, -ang);
      const std::complex<double> w = std::polar(1.0, ang) * std::pow(alpha, (double)j / n) / (double)n;
      const std::complex<double> gv(c->V[2 * e], c->V[2 * e + 1]), gw(c->Vinv[2 * e], c->Vinv[2 * e + 1]);
      vmax = std::max(vmax, std::abs(v));
      imax = std::max(imax, std::abs(w));
      dv = std::max(dv, std::abs(gv - v));
      di = std::max(di, std::abs(gw - w));
    }
  if (!(dv <= 1e-12 * vmax && di <= 1e-12 * imax)) return false;
  *alpha_out = alpha;
  return true;
}

template <typename T>
void alloc_prec(pd_ctx *c) {
  using C = typename Cx<T>::type;
  Prec<T> &P = prec<T>(c);
  const int n = c->n, L = c->L;
  P.lv.resize(L);
  for (int l = 0; l < L; l++) {
    LevelBufs &B = P.lv[l];
    B.N = c->Ns[l];
    B.P = B.N + 1;
    const size_t bytes = (size_t)n * B.N * B.P * sizeof(C);
    B.z[0] = dalloc<void *>(c, bytes);
    B.z[1] = dalloc<void *>(c, bytes);
    B.b = dalloc<void *>(c, bytes);
  }
  if (c->cfg.fused == 2 || (c->cfg.fused == 1 && sizeof(T) == sizeof(float))) {
    const FusedGeom g = fused_geom<T>();
    const int e = (int)(sizeof(C) / 8);
    for (int l = 0; l + 1 < L && l < c->lc; l++) {
      LevelBufs &B = P.lv[l], &Bc = P.lv[l + 1];
      for (int q = 0; q < 2; q++) {
        B.sr_z[q] = grid_map(c, B.z[q], B.N, B.P, n, e, g.sr_zw, g.sr_zh);
        B.ps_z[q] = grid_map(c, B.z[q], B.N, B.P, n, e, g.ps_zw, g.ps_zh);
        B.ps_e[q] = grid_map(c, Bc.z[q], Bc.N, Bc.P, n, e, g.ps_ew, g.ps_eh);
      }
      B.sr_b = grid_map(c, B.b, B.N, B.P, n, e, g.sr_bw, g.sr_bh);
      B.ps_b = grid_map(c, B.b, B.N, B.P, n, e, g.ps_bw, g.ps_bh);
      B.maps = true;
    }
    ck(c, prepare_fused<T>());
    ck(c, prepare_stream<T>());
    c->stream_grid = stream_grid<T>(c->num_sms);
  }
  // smoother coefficients in the scaled form of pd_internal.h
  std::vector<Coef<T>> cf((size_t)L * n);
  for (int l = 0; l < L; l++) {
    const double h = hl(c, l);
    for (int j = 0; j < n; j++) {
      const std::complex<double> lam =
          std::complex<double>(c->shifts[2 * j], c->shifts[2 * j + 1]) / c->kappa;
      const std::complex<double> eta = lam * h * h, d = 4.0 + eta;
      const double w = c->omega[(size_t)j * L + l];
      double abc[6];
      vanka_abc(eta.real(), eta.imag(), abc);
      std::complex<double> ca, cb, cc;
      if (c->cfg.smoother == 1) {
        ca = w / d;
        cb = cc = 0.0;
      } else {
        ca = w * std::complex<double>(abc[0], abc[1]);
        cb = w * std::complex<double>(abc[2], abc[3]) * 0.5;
        cc = w * std::complex<double>(abc[4], abc[5]) * 0.25;
      }
      Coef<T> &k = cf[(size_t)l * n + j];
      k.d.x = (T)d.real(); k.d.y = (T)d.imag();
      k.ca.x = (T)ca.real(); k.ca.y = (T)ca.imag();
      k.cb.x = (T)cb.real(); k.cb.y = (T)cb.imag();
      k.cc.x = (T)cc.real(); k.cc.y = (T)cc.imag();
    }
  }
  P.coef = dalloc<Coef<T> *>(c, cf.size() * sizeof(Coef<T>));
  ck(c, cudaMemcpy(P.coef, cf.data(), cf.size() * sizeof(Coef<T>), cudaMemcpyHostToDevice));
  // inverse of the scaled coarsest matrix h^2 L_j = (4 + eta) I - (neighbours)
  const int Nc = c->Ns[L - 1], m = Nc * Nc;
  const double h = hl(c, L - 1);
  std::vector<C> inv((size_t)n * m * m);
  for (int j = 0; j < n; j++) {
    const std::complex<double> lam =
        std::complex<double>(c->shifts[2 * j], c->shifts[2 * j + 1]) / c->kappa;
    const std::complex<double> d = 4.0 + lam * h * h;
    std::vector<double> A((size_t)2 * m * m, 0.0);
    for (int i = 0; i < Nc; i++)
      for (int q = 0; q < Nc; q++) {
        const int p = i * Nc + q;
        A[2 * ((size_t)p * m + p)] = d.real();
        A[2 * ((size_t)p * m + p) + 1] = d.imag();
        if (i > 0) A[2 * ((size_t)p * m + p - Nc)] = -1.0;
        if (i < Nc - 1) A[2 * ((size_t)p * m + p + Nc)] = -1.0;
        if (q > 0) A[2 * ((size_t)p * m + p - 1)] = -1.0;
        if (q < Nc - 1) A[2 * ((size_t)p * m + p + 1)] = -1.0;
      }
    if (invert_dense(m, A) != 0) throw PD_ERR_SING;
    for (size_t e = 0; e < (size_t)m * m; e++) {
      inv[(size_t)j * m * m + e].x = (T)A[2 * e];
      inv[(size_t)j * m * m + e].y = (T)A[2 * e + 1];
    }
  }
  P.cinv = dalloc<C *>(c, inv.size() * sizeof(C));
  ck(c, cudaMemcpy(P.cinv, inv.data(), inv.size() * sizeof(C), cudaMemcpyHostToDevice));
  if (c->have_V) {
    std::vector<C> wf((size_t)n * n), wi((size_t)n * n);
    for (size_t e = 0; e < (size_t)n * n; e++) {
      wf[e].x = (T)c->Vinv[2 * e];
      wf[e].y = (T)c->Vinv[2 * e + 1];
      wi[e].x = (T)c->V[2 * e];
      wi[e].y = (T)c->V[2 * e + 1];
    }
    P.Wf = dalloc<C *>(c, wf.size() * sizeof(C));
    P.Wi = dalloc<C *>(c, wi.size() * sizeof(C));
    ck(c, cudaMemcpy(P.Wf, wf.data(), wf.size() * sizeof(C), cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.Wi, wi.data(), wi.size() * sizeof(C), cudaMemcpyHostToDevice));
  }
  double alpha_fft = 0.0;
  if (c->have_V && c->cfg.fft_transforms && fft_transforms_supported(n) &&
      alpha_circulant_alpha(c, &alpha_fft)) {
    std::vector<T> wf(n), wf1(n), wi(n);
    std::vector<C> twf(n), twi(n);
    const double h0 = hl(c, 0);
    for (int k = 0; k < n; k++) {
      const double a = std::pow(alpha_fft, (double)k / n);
      wf[k] = (T)(a * h0 * h0 / (c->kappa * n));
      wf1[k] = (T)(a / n);
      wi[k] = (T)(1.0 / a);
      const std::complex<double> e = std::polar(1.0, 2.0 * M_PI * k / n);
      twf[k].x = (T)e.real();
      twf[k].y = (T)e.imag();
      twi[k].x = (T)e.real();
      twi[k].y = (T)-e.imag();
    }
    P.fft_wf = dalloc<T *>(c, n * sizeof(T));
    P.fft_wf1 = dalloc<T *>(c, n * sizeof(T));
    P.fft_wi = dalloc<T *>(c, n * sizeof(T));
    P.fft_twf = dalloc<C *>(c, n * sizeof(C));
    P.fft_twi = dalloc<C *>(c, n * sizeof(C));
    ck(c, cudaMemcpy(P.fft_wf, wf.data(), n * sizeof(T), cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.fft_wf1, wf1.data(), n * sizeof(T), cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.fft_wi, wi.data(), n * sizeof(T), cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.fft_twf, twf.data(), n * sizeof(C), cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.fft_twi, twi.data(), n * sizeof(C), cudaMemcpyHostToDevice));
    ck(c, prepare_fft_transforms<T>());
    P.fft = true;
  }
  if (!P.fft && sizeof(T) == sizeof(float) && c->have_V && c->cfg.tensor_transforms &&
      tc_transforms_supported(c->N, n)) {
    const size_t fa = tc_operand_floats(n, false), ia = tc_operand_floats(n, true);
    std::vector<float> fh(fa), fl(fa), ih(ia), il(ia), f1h(fa), f1l(fa), ih2(ia), il2(ia);
    const double h0 = hl(c, 0);
    tc_build_operands(n, c->Vinv.data(), c->V.data(), h0 * h0 / c->kappa, fh.data(), fl.data(), ih.data(),
                      il.data());
    tc_build_operands(n, c->Vinv.data(), c->V.data(), 1.0, f1h.data(), f1l.data(), ih2.data(), il2.data());
    P.tc_fwd_hi = dalloc<float *>(c, fa * 4);
    P.tc_fwd_lo = dalloc<float *>(c, fa * 4);
    P.tc_fwd1_hi = dalloc<float *>(c, fa * 4);
    P.tc_fwd1_lo = dalloc<float *>(c, fa * 4);
    P.tc_inv_hi = dalloc<float *>(c, ia * 4);
    P.tc_inv_lo = dalloc<float *>(c, ia * 4);
    ck(c, cudaMemcpy(P.tc_fwd_hi, fh.data(), fa * 4, cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.tc_fwd_lo, fl.data(), fa * 4, cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.tc_fwd1_hi, f1h.data(), fa * 4, cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.tc_fwd1_lo, f1l.data(), fa * 4, cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.tc_inv_hi, ih.data(), ia * 4, cudaMemcpyHostToDevice));
    ck(c, cudaMemcpy(P.tc_inv_lo, il.data(), ia * 4, cudaMemcpyHostToDevice));
    ck(c, prepare_tc_transforms());
    ck(c, tc_launch_grid(c->num_sms, n, false, &P.tc_grid_fwd));
    ck(c, tc_launch_grid(c->num_sms, n, true, &P.tc_grid_inv));
    P.tc = true;
  }
  // the attributes are per kernel, shared by all contexts: set the largest any context
  // can use (coarse launches never exceed kCoarseSmemLimit; transforms need n <= 128)
  ck(c, prepare_coarse<T>(kCoarseSmemLimit));
  ck(c, prepare_transforms<T>(kMaxShifts));
  if (P.lv.size() > 0 && P.lv[0].maps) autotune_fused<T>(c);
}

template <typename T>
void run_cycle(pd_ctx *c, int l, bool zzero, bool top, const int *active, double tol, int maxit);

// The same cycle with the last pre-smoothing step fused with residual and restriction
// and the interpolation fused with the first post-smoothing step (fused_kernels.cu).
template <typename T>
void run_cycle_fused(pd_ctx *c, int l, bool zzero, bool top, const int *active, double tol,
                     int maxit) {
  Prec<T> &P = prec<T>(c);
  LevelBufs &B = P.lv[l], &Bc = P.lv[l + 1];
  const int N = B.N, n = c->n;
  const View b = view(B.b, N, B.P);
  View z[2] = {view(B.z[0], N, B.P), view(B.z[1], N, B.P)};
  const Coef<T> *cf = P.coef + (size_t)l * n;
  const bool jac = c->cfg.smoother == 1;
  int &cur = c->cur[l];
  const double w = sizeof(typename Cx<T>::type), pts = (double)N * N, ptsc = (double)Bc.N * Bc.N;
  const FusedGeom g = fused_geom<T>();
  const int ftiles = fused_tiles(N, g.TX, g.TY);
  const int grid = std::max(1, std::min(c->num_sms, n * ftiles));
  int *err = c->st.flags;
  bool norm = top;
  for (int s = 0; s + 1 < c->cfg.nu1; s++) {
    PD_PROF(l == 0 ? PD_KC_SMOOTH0 : PD_KC_SMOOTH_C, (zzero ? 2 : 3) * w * pts, norm ? 1 : 2,
            launch_smooth<T>(c->stream, N, n, z[cur], z[cur ^ 1], b, (T)1, cf, active, zzero, jac,
                             norm ? c->st.partials : nullptr, c->st.max_tiles));
    ck_launch(c);
    if (norm) {
      PD_PROF(PD_KC_CONVERGE, 8.0 * smooth_tiles(N), 1,
              launch_converge(c->stream, n, smooth_tiles(N), c->st, tol, maxit, c->stall, cur));
      ck_launch(c);
      norm = false;
    }
    cur ^= 1;
    zzero = false;
  }
  const bool streams = B.variant == 2;
  const int units = streams ? stream_units(N, B.seg) : ftiles;
  if (streams)
    PD_PROF(l == 0 ? PD_KC_SR0 : PD_KC_SR_C, (zzero ? 2 : 3) * w * pts + w * ptsc, norm ? 1 : 2,
            launch_sr_stream<T>(c->stream, c->stream_grid, N, n, B.seg, z[cur], b, z[cur ^ 1],
                                view(Bc.b, Bc.N, Bc.P), cf, active, zzero,
                                norm ? c->st.partials : nullptr, c->st.max_tiles));
  else
    PD_PROF(l == 0 ? PD_KC_SR0 : PD_KC_SR_C, (zzero ? 2 : 3) * w * pts + w * ptsc, norm ? 1 : 2,
            launch_smooth_restrict<T>(c->stream, grid, B.sr_z[cur], B.sr_b, N, n, z[cur ^ 1],
                                      view(Bc.b, Bc.N, Bc.P), cf, active, zzero,
                                      norm ? c->st.partials : nullptr, c->st.max_tiles, err));
  ck_launch(c);
  if (norm) {
    PD_PROF(PD_KC_CONVERGE, 8.0 * units, 1,
            launch_converge(c->stream, n, units, c->st, tol, maxit, c->stall, cur));
    ck_launch(c);
  }
  cur ^= 1;
  c->cur[l + 1] = 0;
  if (l + 1 >= c->lc) {
    PD_PROF(PD_KC_COARSE, 2 * w * ptsc, 2,
            launch_coarse<T>(c->stream, c->plan, l + 1, n, view(Bc.b, Bc.N, Bc.P), (T)1,
                             view(Bc.z[0], Bc.N, Bc.P), P.coef, P.cinv, active, c->cfg.cycle_gamma,
                             0, 0, 0.0, 0, c->st));
    ck_launch(c);
  } else {
    bool zz = true;
    for (int gm = 0; gm < c->cfg.cycle_gamma; gm++) {
      run_cycle<T>(c, l + 1, zz, false, active, tol, maxit);
      zz = false;
    }
  }
  if (streams)
    PD_PROF(l == 0 ? PD_KC_PS0 : PD_KC_PS_C, 3 * w * pts + w * ptsc, 2,
            launch_ps_stream<T>(c->stream, c->stream_grid, N, n, B.seg, z[cur],
                                view(Bc.z[c->cur[l + 1]], Bc.N, Bc.P), b, z[cur ^ 1], cf, active));
  else
    PD_PROF(l == 0 ? PD_KC_PS0 : PD_KC_PS_C, 3 * w * pts + w * ptsc, 2,
            launch_prolong_smooth<T>(c->stream, grid, B.ps_z[cur], B.ps_e[c->cur[l + 1]], B.ps_b, N,
                                     n, z[cur ^ 1], cf, active, err));
  ck_launch(c);
  cur ^= 1;
  for (int s = 1; s < c->cfg.nu2; s++) {
    PD_PROF(l == 0 ? PD_KC_SMOOTH0 : PD_KC_SMOOTH_C, 3 * w * pts, 2,
            launch_smooth<T>(c->stream, N, n, z[cur], z[cur ^ 1], b, (T)1, cf, active, false, jac,
                             nullptr, 0));
    ck_launch(c);
    cur ^= 1;
  }
}

// ---- one cycle on the global-memory levels (Sec. 3), recursing to the coarse kernel ----
template <typename T>
void run_cycle(pd_ctx *c, int l, bool zzero, bool top, const int *active, double tol, int maxit) {
  Prec<T> &P = prec<T>(c);
  LevelBufs &B = P.lv[l];
  const int N = B.N, n = c->n;
  const View b = view(B.b, N, B.P);
  View z[2] = {view(B.z[0], N, B.P), view(B.z[1], N, B.P)};
  const Coef<T> *cf = P.coef + (size_t)l * n;
  const bool jac = c->cfg.smoother == 1;
  int &cur = c->cur[l];
  const double w = sizeof(typename Cx<T>::type), pts = (double)N * N;
  const int ks = l == 0 ? PD_KC_SMOOTH0 : PD_KC_SMOOTH_C;
  if (l >= c->lc) {
    PD_PROF(PD_KC_COARSE, (zzero ? 2 : 3) * w * pts, 2,
            launch_coarse<T>(c->stream, c->plan, l, n, b, (T)1, z[cur], P.coef, P.cinv, active, 1,
                             zzero ? 0 : 1, 0, 0.0, 0, c->st));
    ck_launch(c);
    return;
  }
  if (B.maps && c->cfg.nu1 >= 1 && c->cfg.nu2 >= 1) {
    run_cycle_fused<T>(c, l, zzero, top, active, tol, maxit);
    return;
  }
  int s = 0;
  if (top) {
    if (c->cfg.nu1 >= 1) {
      PD_PROF(ks, (zzero ? 2 : 3) * w * pts, 1,
              launch_smooth<T>(c->stream, N, n, z[cur], z[cur ^ 1], b, (T)1, cf, active, zzero, jac,
                               c->st.partials, c->st.max_tiles));
      PD_PROF(PD_KC_CONVERGE, 8.0 * smooth_tiles(N), 1,
              launch_converge(c->stream, n, smooth_tiles(N), c->st, tol, maxit, c->stall, cur));
      ck_launch(c, 2);
      cur ^= 1;
      zzero = false;
      s = 1;
    } else {
      PD_PROF(ks, (zzero ? 1 : 2) * w * pts, 1,
              launch_resnorm<T>(c->stream, N, n, z[cur], b, (T)1, cf, active, zzero,
                                c->st.partials, c->st.max_tiles));
      PD_PROF(PD_KC_CONVERGE, 8.0 * smooth_tiles(N), 1,
              launch_converge(c->stream, n, smooth_tiles(N), c->st, tol, maxit, c->stall, cur));
      ck_launch(c, 2);
    }
  }
  for (; s < c->cfg.nu1; s++) {
    PD_PROF(ks, (zzero ? 2 : 3) * w * pts, 2,
            launch_smooth<T>(c->stream, N, n, z[cur], z[cur ^ 1], b, (T)1, cf, active, zzero, jac,
                             nullptr, 0));
    ck_launch(c);
    cur ^= 1;
    zzero = false;
  }
  LevelBufs &Bc = P.lv[l + 1];
  const double ptsc = (double)Bc.N * Bc.N;
  PD_PROF(l == 0 ? PD_KC_RESTRICT0 : PD_KC_RESTRICT_C, (zzero ? 1 : 2) * w * pts + w * ptsc, 2,
          launch_residual_restrict<T>(c->stream, N, n, z[cur], b, (T)1, view(Bc.b, Bc.N, Bc.P),
                                      (T)1, cf, active, zzero));
  ck_launch(c);
  c->cur[l + 1] = 0;
  if (l + 1 >= c->lc) {
    PD_PROF(PD_KC_COARSE, 2 * w * ptsc, 2,
            launch_coarse<T>(c->stream, c->plan, l + 1, n, view(Bc.b, Bc.N, Bc.P), (T)1,
                             view(Bc.z[0], Bc.N, Bc.P), P.coef, P.cinv, active, c->cfg.cycle_gamma,
                             0, 0, 0.0, 0, c->st));
    ck_launch(c);
  } else {
    bool zz = true;
    for (int g = 0; g < c->cfg.cycle_gamma; g++) {
      run_cycle<T>(c, l + 1, zz, false, active, tol, maxit);
      zz = false;
    }
  }
  if (zzero) {
    ck(c, cudaMemsetAsync(z[cur].p, 0, (size_t)n * z[cur].plane * sizeof(typename Cx<T>::type),
                          c->stream));
  }
  PD_PROF(l == 0 ? PD_KC_PROLONG0 : PD_KC_PROLONG_C, 2 * w * pts + w * ptsc, 2,
          launch_prolong_add<T>(c->stream, N, n, z[cur], view(Bc.z[c->cur[l + 1]], Bc.N, Bc.P),
                                active));
  ck_launch(c);
  for (s = 0; s < c->cfg.nu2; s++) {
    PD_PROF(ks, 3 * w * pts, 2,
            launch_smooth<T>(c->stream, N, n, z[cur], z[cur ^ 1], b, (T)1, cf, active, false, jac,
                             nullptr, 0));
    ck_launch(c);
    cur ^= 1;
  }
}

// One cycle of level 0 as a CUDA graph: captured the first time its key is seen, then
// replayed; the host-side ping-pong state a captured cycle leaves is restored on every
// replay.  Returns false (nothing launched) where graphs do not apply or a capture fails.
template <typename T>
bool cycle_graph(pd_ctx *c, bool zzero, double tol, int cmax) {
  if (!c->cfg.cuda_graphs || c->prof_on || !c->graphs_ok || c->stream == nullptr) return false;
  const int prec_id = sizeof(T) == sizeof(double) ? 0 : 1;
  for (const auto &g : c->graphs)
    if (g.prec == prec_id && g.zzero == (int)zzero && g.cur0 == c->cur[0] && g.cmax == cmax &&
        g.tol == tol && g.stall == c->stall) {
      ck(c, cudaGraphLaunch(g.exec, c->stream));
      std::memcpy(c->cur, g.cur_after, sizeof(c->cur));
      c->launches += g.launches;
      return true;
    }
  if (c->graphs.size() >= 32) return false;
  pd_ctx::CycleGraph g{};
  g.prec = prec_id;
  g.zzero = zzero;
  g.cur0 = c->cur[0];
  g.cmax = cmax;
  g.tol = tol;
  g.stall = c->stall;
  int cur_before[kMaxLevels];
  std::memcpy(cur_before, c->cur, sizeof(c->cur));
  const long long l0 = c->launches;
  auto give_up = [&](cudaGraph_t gr) {
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    std::memcpy(c->cur, cur_before, sizeof(c->cur));
    c->launches = l0;
    c->graphs_ok = false;
    return false;
  };
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return give_up(nullptr);
  cudaGraph_t graph = nullptr;
  try {
    run_cycle<T>(c, 0, zzero, true, c->st.active, tol, cmax);
  } catch (const CudaFail &) {
    cudaStreamEndCapture(c->stream, &graph);
    return give_up(graph);
  }
  if (cudaStreamEndCapture(c->stream, &graph) != cudaSuccess || !graph) return give_up(graph);
  if (cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) return give_up(graph);
  cudaGraphDestroy(graph);
  std::memcpy(g.cur_after, c->cur, sizeof(c->cur));
  g.launches = c->launches - l0;
  c->graphs.push_back(g);
  ck(c, cudaGraphLaunch(g.exec, c->stream));
  return true;
}

// Solve of eq. (2) for all shifts with the right-hand side already in lv[0].b
// (scaled by h^2), in three parts so that several contexts can advance together:
// solve_begin resets the state (returns the cycle limit, or -1 when the coarse kernel
// solved the whole problem), solve_cycle queues cycle `cyc` and the copy of its active
// count, solve_poll waits for the count of the cycle before (false once it left no shift
// active), solve_end collects the answers.  On return the per-shift answers are in
// lv[0].z[final_buf[j]], and h_iters/h_relres (pinned copies) hold cycles and relative
// residuals.  skip_final: after the last permitted cycle stop without computing the
// residual of the last iterate (the refinement evaluates its own residual anyway).
template <typename T>
int solve_begin(pd_ctx *c, double tol, int maxit, double stall) {
  Prec<T> &P = prec<T>(c);
  c->stall = stall;
  LevelBufs &B = P.lv[0];
  const int n = c->n;
  const double w = sizeof(typename Cx<T>::type), pts = (double)B.N * B.N;
  PD_PROF(PD_KC_OTHER, 0.0, 0, launch_reset_state(c->stream, n, c->st));
  ck_launch(c);
  if (c->lc == 0) {
    PD_PROF(PD_KC_COARSE, 2 * w * pts, 0,
            launch_coarse<T>(c->stream, c->plan, 0, n, view(B.b, B.N, B.P), (T)1,
                             view(B.z[0], B.N, B.P), P.coef, P.cinv, nullptr, 0, 0, 1, tol, maxit,
                             c->st));
    ck_launch(c);
    return -1;
  }
  ck(c, cudaMemsetAsync(B.z[0], 0, (size_t)n * B.N * B.P * sizeof(typename Cx<T>::type),
                        c->stream));
  c->cur[0] = 0;
  return std::min(maxit, std::max(c->cfg.maxit, c->cfg.inner_maxit));
}

template <typename T>
void solve_cycle(pd_ctx *c, int cyc, int cmax, double tol, bool skip_final) {
  c->cur_cyc = cyc;
  if (skip_final && cyc == cmax && cyc > 0) {
    PD_PROF(PD_KC_OTHER, 0.0, 0, launch_finalize(c->stream, c->n, c->st, c->cur[0]));
    ck_launch(c);
  } else if (!cycle_graph<T>(c, cyc == 0, tol, cmax)) {
    run_cycle<T>(c, 0, cyc == 0, true, c->st.active, tol, cmax);
  }
  ck(c, cudaMemcpyAsync(&c->h_hist[cyc], c->st.nactive, sizeof(int), cudaMemcpyDeviceToHost,
                        c->stream));
  ck(c, cudaEventRecord(c->ev[cyc & 1], c->stream));
}

bool solve_poll(pd_ctx *c, int cyc) {
  if (cyc < 1) return true;
  ck(c, cudaEventSynchronize(c->ev[(cyc - 1) & 1]));
  return c->h_hist[cyc - 1] != 0;
}

template <typename T>
pd_status solve_end(pd_ctx *c, double tol) {
  const int n = c->n;
  ck(c, cudaMemcpyAsync(c->h_iters, c->st.iters, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  ck(c, cudaMemcpyAsync(c->h_relres, c->st.relres, n * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream));
  ck(c, cudaMemcpyAsync(&c->h_pinned[2], c->st.flags, sizeof(int), cudaMemcpyDeviceToHost,
                        c->stream));
  ck(c, cudaStreamSynchronize(c->stream));
  prof_resolve(c);
  c->cur_cyc = -1;
  if (c->h_pinned[2] & 2) {
    c->err = "a bounded TMA wait ran out in a fused kernel";
    throw CudaFail{cudaErrorLaunchTimeout};
  }
  if (c->h_pinned[2] & 1) return PD_ERR_NAN;
  for (int j = 0; j < n; j++)
    if (!(c->h_relres[j] <= tol)) return PD_ERR_NOCONV;
  return PD_OK;
}

template <typename T>
pd_status solve_levels(pd_ctx *c, double tol, int maxit, double stall = 0.0, bool skip_final = false) {
  const int cmax = solve_begin<T>(c, tol, maxit, stall);
  for (int cyc = 0; cyc <= cmax; cyc++) {
    solve_cycle<T>(c, cyc, cmax, tol, skip_final);
    if (!solve_poll(c, cyc)) break;
  }
  return solve_end<T>(c, tol);
}

// Several contexts solved together: every round queues one cycle of each context still
// iterating (each on its own stream), then waits for the counts of the round before.
// inner: the refinement's inner solve (inner_tol, inner_maxit, stall_ratio, no final
// residual) instead of the plain one (tol, maxit).
template <typename T>
void lockstep_solve(const std::vector<pd_ctx *> &cs, bool inner, std::vector<pd_status> &rc) {
  const size_t k = cs.size();
  std::vector<int> cmax(k);
  std::vector<char> live(k), sent(k);
  auto tol_of = [&](pd_ctx *c) { return inner ? c->cfg.inner_tol : c->cfg.tol; };
  for (size_t i = 0; i < k; i++) {
    pd_ctx *c = cs[i];
    cmax[i] = solve_begin<T>(c, tol_of(c), inner ? c->cfg.inner_maxit : c->cfg.maxit,
                             inner ? c->cfg.stall_ratio : 0.0);
    live[i] = cmax[i] >= 0;
  }
  for (int cyc = 0;; cyc++) {
    bool any = false;
    for (size_t i = 0; i < k; i++) {
      sent[i] = live[i] && cyc <= cmax[i];
      if (sent[i]) {
        solve_cycle<T>(cs[i], cyc, cmax[i], tol_of(cs[i]), inner);
        any = true;
      } else {
        live[i] = 0;
      }
    }
    if (!any) break;
    for (size_t i = 0; i < k; i++)
      if (sent[i] && !solve_poll(cs[i], cyc)) live[i] = 0;
  }
  rc.assign(k, PD_OK);
  for (size_t i = 0; i < k; i++) rc[i] = solve_end<T>(cs[i], tol_of(cs[i]));
}

// x as a float-float pair: hi = x rounded to FP32, lo = the rest rounded to FP32
float2 split_ff(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// A sum of squares of `count` values scaled by a power of two is trusted when the rms of
// the scaled values lies in [2^-24, 2^24]: no square is near the FP32 underflow or
// overflow.  rescale: the exponent that brings that rms to about 1 (48 bits down when the
// sum is not finite: an FP32 square overflowed, which the float-float sums turn into NaN,
// or the data hold NaN/Inf; 48 bits up when every square underflowed or the data are 0).
bool scale_fits(double sum, double count) {
  if (!(sum > 0.0) || !std::isfinite(sum)) return false;
  const double rms = std::sqrt(sum / count);
  return rms >= 0x1p-24 && rms <= 0x1p24;
}
int rescale(double sum, double count, int sig) {
  int s;
  if (!std::isfinite(sum)) s = sig - 48;
  else if (!(sum > 0.0)) s = sig + 48;
  else s = sig - (int)std::lround(0.5 * std::log2(sum / count));
  return std::max(-120, std::min(120, s));
}

// ---- FP64 refinement of the shifted systems around the FP32 multigrid ----
struct RefRun {
  pd_ctx *c = nullptr;
  double2 *z = nullptr;
  const double2 *b = nullptr;
  std::vector<double> bn, prev, relres;
  std::vector<int> it_sum, sig;  // sig[j]: the shift's FP32 right-hand side is 2^sig[j] r_j
  int evals = 0;  // residual evaluations done (the first one is ||b||)
  bool done = false;
  pd_status rc = PD_OK;
};

// queues r = b - L z (z = 0 on the first evaluation) into the FP32 level-0 RHS, each
// shift's times 2^sig[j], its per-shift partial norms and their copy to the host
void refine_eval_launch(RefRun &r) {
  pd_ctx *c = r.c;
  LevelBufs &B = c->p32.lv[0];
  const int N = c->N, n = c->n, gx = shift_residual_blocks(N, n, c->num_sms);
  const bool first = r.evals == 0;
  const double h = hl(c, 0);
  const double w = 8.0, m = (double)N * N;
  if ((int)r.sig.size() != n) r.sig.assign(n, 0);  // a new run; retries keep their scales
  for (int j = 0; j < n; j++) c->h_rsc[j] = std::ldexp(1.0f, r.sig[j]);
  ck(c, cudaMemcpyAsync(c->d_rsc, c->h_rsc, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  if (!first && c->cfg.fx_residual)  // without FP64 arithmetic (the first one is r = b)
    PD_PROF(PD_KC_RESIDUAL, (32.0 + w) * m, 0,
            launch_shift_residual_fx(c->stream, gx, N, n, r.z, r.b, c->d_lam, c->kappa / (h * h),
                                     (float)rs(c, 0), c->d_rsc, view(B.b, N, B.P), c->d_frozen,
                                     c->d_srpart));
  else
    PD_PROF(PD_KC_RESIDUAL, (first ? 16.0 + w : 32.0 + w) * m, 0,
            launch_shift_residual(c->stream, gx, N, n, first ? nullptr : r.z, r.b, c->d_c1,
                                  c->kappa / (h * h), (float)rs(c, 0), c->d_rsc, view(B.b, N, B.P),
                                  first ? nullptr : c->d_frozen, first, c->d_srpart));
  ck_launch(c, !first && c->cfg.fx_residual ? 2 : 1);  // the fx residual: interior and edge kernels
  ck(c, cudaMemcpyAsync(c->h_srpart, c->d_srpart, (first ? 2 : 1) * (size_t)n * gx * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream));
  ck(c, cudaEventRecord(c->ev[0], c->stream));
}

// after the evaluation: relative residuals; shifts that converged, stopped contracting or
// used up max_refine corrections are frozen (their next RHS is zero and they get no
// update).  A shift whose scaled residual fell outside the trusted range (scale_fits) gets
// a corrected scale and the evaluation is repeated (at most three times).  Sets r.done
// when no shift needs another correction.
void refine_eval_finish(RefRun &r) {
  pd_ctx *c = r.c;
  const int N = c->N, n = c->n, gx = shift_residual_blocks(N, n, c->num_sms);
  const double m = (double)N * N;
  const bool first = r.evals == 0;
  std::vector<double> sr(n), sb(n);
  for (int tries = 0;; tries++) {
    ck(c, cudaEventSynchronize(c->ev[0]));
    prof_resolve(c);
    bool again = false;
    for (int j = 0; j < n; j++) {
      if (!first && c->h_frozen[j]) continue;
      double s = 0.0, b = 0.0;
      for (int x = 0; x < gx; x++) s += c->h_srpart[(size_t)j * gx + x];
      if (first)
        for (int x = 0; x < gx; x++) b += c->h_srpart[(size_t)(n + j) * gx + x];
      sr[j] = s;
      sb[j] = b;
      if (tries >= 3 || scale_fits(s, m)) continue;
      if (first) {
        if (!(b > 0.0) || !std::isfinite(b)) continue;  // b_j = 0 or not finite: nothing to scale
        r.sig[j] = std::max(-120, std::min(120, -(int)std::lround(0.5 * std::log2(b / m))));
      } else {
        r.sig[j] = rescale(s, m, r.sig[j]);
      }
      again = true;
    }
    if (!again) break;
    refine_eval_launch(r);
  }
  if (first) {
    r.bn.assign(n, 0.0);
    r.prev.assign(n, 0.0);
    r.relres.assign(n, 1.0);
    r.it_sum.assign(n, 0);
    for (int j = 0; j < n; j++) c->h_frozen[j] = 0;
  }
  bool any = false;
  for (int j = 0; j < n; j++) {
    if (c->h_frozen[j]) continue;
    if (first) r.bn[j] = std::sqrt(sb[j]);
    const double rn = std::sqrt(sr[j]) * std::ldexp(1.0, -r.sig[j]);
    const double rr = !(std::isfinite(rn) && std::isfinite(r.bn[j])) ? std::nan("")
                      : r.bn[j] > 0.0 ? rn / r.bn[j] : 0.0;
    r.relres[j] = rr;
    if (!std::isfinite(rr)) {
      r.rc = PD_ERR_NAN;
      c->h_frozen[j] = 1;
      continue;
    }
    const bool stuck = r.evals >= 2 && rr > 0.9 * r.prev[j];
    if (rr <= c->cfg.tol || stuck || r.evals >= c->cfg.max_refine) c->h_frozen[j] = 1;
    else any = true;
    r.prev[j] = rr;
    // predicted scale of the next residual (a correction reduces it about 30-fold)
    r.sig[j] = std::min(120, r.sig[j] + 5);
  }
  r.evals++;
  ck(c, cudaMemcpyAsync(c->d_frozen, c->h_frozen, n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  r.done = !any || r.rc != PD_OK;
}

// ---- batches of uneven instances: one launch per multigrid level over all instances ----
//
// With V(1,1) cycles of FP32 warp-stream kernels on every global level, a cycle of all
// instances is 2 G + 2 launches (G = the most global levels of an instance), aligned at
// the finest level: the smoothing + restriction of level s of every instance that has it,
// the convergence test of all shifts after level 0, the coarse levels of all instances
// (one CTA per shift), then the interpolation + smoothing of level s for s = G-1 .. 0.
// The tasks (views, coefficient tables, states) are tables in device memory built once;
// a cycle is captured as one CUDA graph per kind and replayed.
struct BatchPlan {
  std::vector<pd_ctx *> ctx;   // every instance
  std::vector<pd_ctx *> cyc;   // those with global levels (the others solve inside k_coarse)
  cudaStream_t stream = nullptr;
  bool ok = false;
  int gmax = 0, total = 0, grid = 0;
  size_t coarse_smem = 0;
  std::vector<int> sr_off, sr_cnt, sr_units, ps_off, ps_cnt, ps_units;
  StreamTask<float> *d_stream = nullptr;
  CoarseTask<float> *d_coarse = nullptr;
  ConvTask *d_conv = nullptr;
  int *d_bnact = nullptr, *h_bnact = nullptr;  // active shifts of all instances (pinned [cycles + 2])
  int *h_total = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<char> zeroed;  // level-0 RHS of a finished instance already cleared
  std::vector<cudaEvent_t> join;  // per instance: its stream's work before the batched cycles
  cudaEvent_t done = nullptr;     // the batched cycles, for the instances' streams
  struct Graph {
    int zzero, cmax;
    double tol, stall;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  bool graphs_ok = true;
  long long launches = 0;
  std::vector<void *> allocs;
};

void free_plan(BatchPlan &bp) {
  for (auto &g : bp.graphs) cudaGraphExecDestroy(g.exec);
  bp.graphs.clear();
  for (void *q : bp.allocs) cudaFree(q);
  bp.allocs.clear();
  if (bp.h_bnact) cudaFreeHost(bp.h_bnact);
  if (bp.h_total) cudaFreeHost(bp.h_total);
  bp.h_bnact = bp.h_total = nullptr;
  for (int k = 0; k < 2; k++)
    if (bp.ev[k]) cudaEventDestroy(bp.ev[k]);
  bp.ev[0] = bp.ev[1] = nullptr;
  for (cudaEvent_t e : bp.join)
    if (e) cudaEventDestroy(e);
  bp.join.clear();
  if (bp.done) cudaEventDestroy(bp.done);
  bp.done = nullptr;
}

// Builds the task tables; leaves bp.ok false (launches instance by instance) unless every
// instance runs FP32 V(1,1) cycles with warp-stream kernels on at least one global level.
void build_plan(BatchPlan &bp) {
  bp.ok = false;
  bp.cyc.clear();
  if (bp.ctx.empty()) return;
  for (pd_ctx *c : bp.ctx) {
    const pd_config &cf = c->cfg;
    if (cf.precision != 1 || cf.nu1 != 1 || cf.nu2 != 1 || cf.cycle_gamma != 1) return;
    if (c->lc < 1) continue;  // the whole solve runs in k_coarse at solve_begin
    for (int l = 0; l < c->lc; l++)
      if (!c->p32.lv[l].maps || c->p32.lv[l].variant != 2) return;
    bp.gmax = std::max(bp.gmax, c->lc);
    bp.cyc.push_back(c);
  }
  pd_ctx *c0 = bp.ctx[0];
  std::vector<StreamTask<float>> st;
  for (int pass = 0; pass < 2; pass++)
    for (int sl = 0; sl < bp.gmax; sl++) {
      (pass == 0 ? bp.sr_off : bp.ps_off).push_back((int)st.size());
      int units = 0, cnt = 0;
      for (pd_ctx *c : bp.cyc) {
        if (c->lc <= sl) continue;
        const LevelBufs &B = c->p32.lv[sl], &Bc = c->p32.lv[sl + 1];
        StreamTask<float> t{};
        t.N = B.N;
        t.n = c->n;
        t.seg = B.seg;
        t.ubegin = units;
        t.b = view(B.b, B.N, B.P);
        t.coef = c->p32.coef + (size_t)sl * c->n;
        t.active = c->st.active;
        if (pass == 0) {
          t.z = view(B.z[0], B.N, B.P);
          t.zout = view(B.z[1], B.N, B.P);
          t.x = view(Bc.b, Bc.N, Bc.P);
          t.partials = sl == 0 ? c->st.partials : nullptr;
          t.part_stride = c->st.max_tiles;
        } else {
          t.z = view(B.z[1], B.N, B.P);
          t.zout = view(B.z[0], B.N, B.P);
          t.x = view(Bc.z[0], Bc.N, Bc.P);
        }
        units += c->n * stream_units(B.N, B.seg);
        st.push_back(t);
        cnt++;
      }
      (pass == 0 ? bp.sr_cnt : bp.ps_cnt).push_back(cnt);
      (pass == 0 ? bp.sr_units : bp.ps_units).push_back(units);
    }
  std::vector<CoarseTask<float>> co;
  std::vector<ConvTask> cv;
  int j0 = 0;
  for (pd_ctx *c : bp.cyc) {
    const LevelBufs &B = c->p32.lv[c->lc];
    CoarseTask<float> t{};
    t.a.plan = c->plan;
    t.a.n = c->n;
    t.a.start = c->lc;
    t.a.block0 = j0;
    t.a.coef = c->p32.coef;
    t.a.cinv = c->p32.cinv;
    t.b = view(B.b, B.N, B.P);
    t.z = view(B.z[0], B.N, B.P);
    t.active = c->st.active;
    co.push_back(t);
    bp.coarse_smem = std::max(bp.coarse_smem, coarse_smem_bytes<float>(c->plan, c->lc));
    ConvTask k{};
    k.st = c->st;
    k.n = c->n;
    k.ntiles = stream_units(c->N, c->p32.lv[0].seg);
    k.j0 = j0;
    cv.push_back(k);
    j0 += c->n;
  }
  bp.total = j0;
  bp.grid = c0->stream_grid;
  auto upload = [&](const void *src, size_t bytes) {
    void *d = nullptr;
    ck(c0, cudaMalloc(&d, std::max<size_t>(bytes, 16)));
    bp.allocs.push_back(d);
    ck(c0, cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice));
    return d;
  };
  bp.d_stream = static_cast<StreamTask<float> *>(upload(st.data(), st.size() * sizeof(st[0])));
  bp.d_coarse = static_cast<CoarseTask<float> *>(upload(co.data(), co.size() * sizeof(co[0])));
  bp.d_conv = static_cast<ConvTask *>(upload(cv.data(), cv.size() * sizeof(cv[0])));
  {
    void *d = nullptr;
    ck(c0, cudaMalloc(&d, sizeof(int)));
    bp.allocs.push_back(d);
    bp.d_bnact = static_cast<int *>(d);
  }
  const int hist = std::max(c0->cfg.maxit, c0->cfg.inner_maxit) + 2;
  ck(c0, cudaMallocHost(&bp.h_bnact, hist * sizeof(int)));
  ck(c0, cudaMallocHost(&bp.h_total, sizeof(int)));
  for (int k = 0; k < 2; k++) ck(c0, cudaEventCreateWithFlags(&bp.ev[k], cudaEventDisableTiming));
  bp.join.assign(bp.ctx.size(), nullptr);
  for (auto &e : bp.join) ck(c0, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  ck(c0, cudaEventCreateWithFlags(&bp.done, cudaEventDisableTiming));
  bp.zeroed.assign(bp.ctx.size(), 0);
  bp.ok = true;
}

// One cycle of every instance (see BatchPlan).
void plan_cycle(BatchPlan &bp, bool zzero, double tol, int cmax, double stall) {
  pd_ctx *c0 = bp.ctx[0];
  const int k = (int)bp.cyc.size();
  for (int sl = 0; sl < bp.gmax; sl++) {
    // the coarser levels start every cycle from a zero correction
    launch_sr_multi<float>(bp.stream, bp.grid, bp.d_stream + bp.sr_off[sl], bp.sr_cnt[sl], bp.sr_units[sl],
                           sl == 0 ? zzero : true, sl == 0);
    if (sl == 0) launch_converge_multi(bp.stream, bp.d_conv, k, bp.total, tol, cmax, stall, 0, bp.d_bnact);
  }
  launch_coarse_multi<float>(bp.stream, bp.d_coarse, k, bp.total, bp.coarse_smem, 1);
  for (int sl = bp.gmax - 1; sl >= 0; sl--)
    launch_ps_multi<float>(bp.stream, bp.grid, bp.d_stream + bp.ps_off[sl], bp.ps_cnt[sl], bp.ps_units[sl]);
  bp.launches += 2 * bp.gmax + 2;
  ck(c0, cudaGetLastError());
}

// plan_cycle through a CUDA graph per (zzero, tol, cmax, stall), captured the first time
void plan_cycle_graph(BatchPlan &bp, bool zzero, double tol, int cmax, double stall) {
  pd_ctx *c0 = bp.ctx[0];
  if (c0->cfg.cuda_graphs && bp.graphs_ok) {
    for (const auto &g : bp.graphs)
      if (g.zzero == (int)zzero && g.cmax == cmax && g.tol == tol && g.stall == stall) {
        ck(c0, cudaGraphLaunch(g.exec, bp.stream));
        bp.launches += 2 * bp.gmax + 2;
        return;
      }
    if (bp.graphs.size() < 16 &&
        cudaStreamBeginCapture(bp.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaGraph_t graph = nullptr;
      bool fine = true;
      try {
        plan_cycle(bp, zzero, tol, cmax, stall);
      } catch (const CudaFail &) {
        fine = false;
      }
      bp.launches -= 2 * bp.gmax + 2;
      BatchPlan::Graph g{(int)zzero, cmax, tol, stall, nullptr};
      if (cudaStreamEndCapture(bp.stream, &graph) == cudaSuccess && graph && fine &&
          cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess) {
        cudaGraphDestroy(graph);
        bp.graphs.push_back(g);
        ck(c0, cudaGraphLaunch(g.exec, bp.stream));
        bp.launches += 2 * bp.gmax + 2;
        return;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      bp.graphs_ok = false;
    }
  }
  plan_cycle(bp, zzero, tol, cmax, stall);
}

// The inner FP32 solves of the refinement for the instances in `act`, every instance's
// cycle in the same launches on the plan's stream (joined with the instances' own
// streams, on which their residual evaluations and updates run side by side); the others
// get a zero right-hand side, so their shifts stop at the first test.
void plan_solve(BatchPlan &bp, const std::vector<pd_ctx *> &act, std::vector<pd_status> &rc) {
  pd_ctx *c0 = bp.ctx[0];
  int cmax = -1;
  for (size_t i = 0; i < bp.ctx.size(); i++) {
    pd_ctx *c = bp.ctx[i];
    const bool on = std::find(act.begin(), act.end(), c) != act.end();
    if (!on && !bp.zeroed[i]) {
      LevelBufs &B = c->p32.lv[0];
      ck(c, cudaMemsetAsync(B.b, 0, (size_t)c->n * B.N * B.P * sizeof(float2), c->stream));
      bp.zeroed[i] = 1;
    }
    if (on) bp.zeroed[i] = 0;
    cmax = std::max(cmax, solve_begin<float>(c, c->cfg.inner_tol, c->cfg.inner_maxit, c->cfg.stall_ratio));
    ck(c, cudaEventRecord(bp.join[i], c->stream));
    ck(c, cudaStreamWaitEvent(bp.stream, bp.join[i], 0));
  }
  const double tol = c0->cfg.inner_tol, stall = c0->cfg.stall_ratio;
  *bp.h_total = bp.total;
  ck(c0, cudaMemcpyAsync(bp.d_bnact, bp.h_total, sizeof(int), cudaMemcpyHostToDevice, bp.stream));
  for (int cyc = 0; cyc <= cmax; cyc++) {
    if (cyc == cmax && cyc > 0) {
      launch_finalize_multi(bp.stream, bp.d_conv, (int)bp.cyc.size(), bp.total, 0, bp.d_bnact);
      bp.launches++;
      ck(c0, cudaGetLastError());
    } else {
      plan_cycle_graph(bp, cyc == 0, tol, cmax, stall);
    }
    ck(c0, cudaMemcpyAsync(&bp.h_bnact[cyc], bp.d_bnact, sizeof(int), cudaMemcpyDeviceToHost, bp.stream));
    ck(c0, cudaEventRecord(bp.ev[cyc & 1], bp.stream));
    if (cyc >= 1) {
      ck(c0, cudaEventSynchronize(bp.ev[(cyc - 1) & 1]));
      if (bp.h_bnact[cyc - 1] == 0) break;
    }
  }
  ck(c0, cudaEventRecord(bp.done, bp.stream));
  for (pd_ctx *c : bp.ctx) ck(c, cudaStreamWaitEvent(c->stream, bp.done, 0));
  rc.assign(act.size(), PD_OK);
  for (size_t i = 0; i < act.size(); i++) rc[i] = solve_end<float>(act[i], act[i]->cfg.inner_tol);
}

// shifted_solve_refined for a set of runs (one per context), advanced together; with a
// plan (all runs' contexts in it) the inner solves are batched launches
void refine_runs(std::vector<RefRun> &runs, BatchPlan *bp = nullptr) {
  for (auto &r : runs) refine_eval_launch(r);
  for (auto &r : runs) refine_eval_finish(r);
  for (;;) {
    std::vector<pd_ctx *> act;
    std::vector<RefRun *> ar;
    for (auto &r : runs)
      if (!r.done) {
        act.push_back(r.c);
        ar.push_back(&r);
      }
    if (act.empty()) break;
    std::vector<pd_status> rc;
    if (bp && bp->ok) plan_solve(*bp, act, rc);
    else lockstep_solve<float>(act, true, rc);
    for (size_t i = 0; i < ar.size(); i++) {
      RefRun &r = *ar[i];
      pd_ctx *c = r.c;
      if (rc[i] == PD_ERR_NAN) {
        r.rc = PD_ERR_NAN;
        r.done = true;
        continue;
      }
      for (int j = 0; j < c->n; j++) r.it_sum[j] += c->h_iters[j];
      LevelBufs &B = c->p32.lv[0];
      const int N = c->N;
      // the first update writes every shift (z = d; d = 0 for a zero right-hand side)
      PD_PROF(PD_KC_OTHER, 24.0 * N * N, 0,
              launch_shift_update(c->stream, N, c->n, r.z, view(B.z[0], N, B.P),
                                  view(B.z[1], N, B.P), c->st.final_buf,
                                  r.evals > 1 ? c->d_frozen : nullptr, c->d_rsc, r.evals > 1));
      ck_launch(c);
      refine_eval_launch(r);
    }
    for (RefRun *r : ar)
      if (!r->done) refine_eval_finish(*r);
  }
  for (auto &r : runs) {
    if (r.rc != PD_OK) continue;
    for (int j = 0; j < r.c->n; j++)
      if (!(r.relres[j] <= r.c->cfg.tol)) r.rc = PD_ERR_NOCONV;
  }
}

// ||fhat - A u|| and ||fhat|| from the per-CTA partial sums (fixed order):
// r (FP64, may be NULL) or r32 (FP32) = fhat - A u and the norms; with a bidiagonal B
// and known_fn >= 0 the ||fhat|| sums are skipped and known_fn returned
// fcache: 0 none, 1 write fhat (float-float) into the context's cache, 2 read it from there
// sig_r: r32 is written times 2^(*sig_r), the FP32 right-hand side of the next refinement
// step kept near unit size; the sums of squares are those of scaled values, checked
// against scale_fits and recomputed (at most three times) with corrected exponents, the
// last exponent used is returned in *sig_r.  Only the FP32 outputs are scaled.
void allatonce_norms(pd_ctx *c, double *r, const double *u, const double *f, const double *u0,
                     double *rn, double *fn, float *r32 = nullptr, double known_fn = -1.0,
                     int fcache = 0, int *sig_r = nullptr) {
  const double m = (double)c->N * c->N, cnt = m * c->n;
  const bool want_f = known_fn < 0.0;
  const bool fx = c->bidiag && r32 && !r && c->cfg.fx_residual;
  const bool scaled = r32 && !r && c->bidiag;
  int sr = sig_r ? *sig_r : 0, sf = c->fsig;
  double a = 0.0, b = 0.0;
  for (int tries = 0;; tries++) {
    int nb = allatonce_blocks();
    if (fx) {
      nb = residual_fx_blocks(c->num_sms);
      const bool use = fcache && c->d_fcache;
      PD_PROF(PD_KC_RESIDUAL,
              (use && fcache == 1 ? 28.0 : 20.0) * m + (u0 && !(use && fcache == 2) ? 8.0 * m / c->n : 0.0), 0,
              launch_residual_fx(c->stream, nb, c->N, c->n, c->boff, c->ihf, r32, u, f, u0, c->d_kbd,
                                 c->d_ku0, std::ldexp(1.0f, sr), std::ldexp(1.0f, sf), want_f, c->d_part,
                                 use && fcache == 2 ? c->d_fcache : nullptr,
                                 use && fcache == 1 ? c->d_fcache : nullptr));
    } else if (c->bidiag) {
      PD_PROF(PD_KC_RESIDUAL,
              (r ? 24.0 : r32 ? 20.0 : 16.0) * m + (u0 ? 8.0 * m / c->n : 0.0), 0,
              launch_residual_bidiag(c->stream, c->N, c->n, c->boff, c->kappa, r, r32, u, f, u0,
                                     c->d_u0coef, c->d_bd, c->d_bs, want_f, c->d_part,
                                     std::ldexp(1.0, sr)));
    } else {
      PD_PROF(PD_KC_RESIDUAL, (r ? 24.0 : 16.0) * m + (u0 ? 8.0 * m / c->n : 0.0), 0,
              launch_allatonce_residual(c->stream, c->N, c->n, c->kappa, r, u, f, u0, c->d_u0coef,
                                        c->d_Bptr, c->d_Bcol, c->d_Bval, c->d_part));
    }
    ck_launch(c, fx ? 2 : 1);  // the fx residual: interior and edge kernels
    ck(c, cudaMemcpyAsync(c->h_part, c->d_part, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    ck(c, cudaStreamSynchronize(c->stream));
    a = 0.0;
    b = 0.0;
    for (int k = 0; k < nb; k++) {
      a += c->h_part[2 * k];
      b += c->h_part[2 * k + 1];
    }
    prof_resolve(c);
    if (!scaled) break;
    // the ||fhat|| sums are scaled only in the FP64-free kernel
    const bool okr = scale_fits(a, cnt), okf = !(fx && want_f) || scale_fits(b, cnt);
    if ((okr && okf) || tries >= 3) break;
    if (!okr) sr = rescale(a, cnt, sr);
    if (!okf) sf = rescale(b, cnt, sf);
  }
  *rn = scaled ? std::sqrt(a) * std::ldexp(1.0, -sr) : std::sqrt(a);
  if (c->bidiag && !want_f) *fn = known_fn;
  else *fn = fx ? std::sqrt(b) * std::ldexp(1.0, -sf) : std::sqrt(b);
  if (sig_r) *sig_r = sr;
  if (fx && want_f) c->fsig = sf;
  if (scaled && !sig_r && sr != 0) {
    // the caller wants r itself: write it once more unscaled (the norms above stand)
    if (fx)
      launch_residual_fx(c->stream, residual_fx_blocks(c->num_sms), c->N, c->n, c->boff, c->ihf, r32, u,
                         f, u0, c->d_kbd, c->d_ku0, 1.0f, 1.0f, false, c->d_part,
                         fcache == 2 && c->d_fcache ? c->d_fcache : nullptr, nullptr);
    else
      launch_residual_bidiag(c->stream, c->N, c->n, c->boff, c->kappa, nullptr, r32, u, f, u0,
                             c->d_u0coef, c->d_bd, c->d_bs, false, c->d_part, 1.0);
    ck_launch(c, fx ? 2 : 1);
    ck(c, cudaStreamSynchronize(c->stream));
  }
}

// forward transform into view g (scaled: the level-0 h^2 scaling; else unscaled);
// f is FP64, or FP32 when f32 (the refinement residual)
// in_scale (a power of two) multiplies an FP64 input; the FFT route is only given FP64
// input unscaled (FP32 inputs arrive scaled already)
template <typename T>
void transform_forward(pd_ctx *c, View g, const void *f, const double *u0, bool scaled,
                       bool f32 = false, double in_scale = 1.0) {
  Prec<T> &P = prec<T>(c);
  const double h = hl(c, 0);
  if (P.fft) {
    launch_fft_forward<T>(c->stream, c->num_sms, c->N, c->n, g, f, f32, u0, c->d_u0coef,
                          scaled ? P.fft_wf : P.fft_wf1, P.fft_twf);
  } else if (P.tc) {
    launch_tc_forward(c->stream, P.tc_grid_fwd, c->N, c->n, g, f, f32, u0, c->d_u0coef,
                      scaled ? P.tc_fwd_hi : P.tc_fwd1_hi, scaled ? P.tc_fwd_lo : P.tc_fwd1_lo,
                      in_scale, c->st.flags);
  } else {
    launch_transform_forward<T>(c->stream, c->N, c->n, g, f, f32, u0, c->d_u0coef, P.Wf,
                                (scaled ? h * h / c->kappa : 1.0) * in_scale);
  }
}

// dscale (a power of two) multiplies the correction: the inverse of the scale of the FP32
// right-hand side it was solved from
template <typename T>
void transform_inverse(pd_ctx *c, double *u, View z0, View z1, const int *final_buf, bool acc,
                       bool imag, double dscale = 1.0) {
  Prec<T> &P = prec<T>(c);
  if (P.fft)
    launch_fft_inverse<T>(c->stream, c->num_sms, c->N, c->n, u, z0, z1, final_buf, P.fft_wi,
                          P.fft_twi, (T)dscale, acc, imag, c->d_imag);
  else if (P.tc)
    launch_tc_inverse(c->stream, P.tc_grid_inv, c->N, c->n, u, z0, z1, final_buf, P.tc_inv_hi,
                      P.tc_inv_lo, (float)dscale, acc, imag, c->d_imag, c->st.flags);
  else
    launch_transform_inverse<T>(c->stream, c->N, c->n, u, z0, z1, final_buf, P.Wi, (T)dscale, acc,
                                imag, c->d_imag);
}

void check_wait_flags(pd_ctx *c) {
  ck(c, cudaMemcpyAsync(&c->h_pinned[2], c->st.flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  ck(c, cudaStreamSynchronize(c->stream));
  if (c->h_pinned[2] & 6) {
    c->err = "a bounded wait ran out in a TMA or tensor-core kernel";
    cudaMemsetAsync(c->st.flags, 0, sizeof(int), c->stream);  // report each timeout once
    throw CudaFail{cudaErrorLaunchTimeout};
  }
}

// relative residual ||r|| / ||fhat||; NaN when either norm is not finite (a NaN or Inf in
// the data), 0 for a zero right-hand side
double rel_of(double rn, double fn) {
  if (!std::isfinite(rn) || !std::isfinite(fn)) return std::nan("");
  return fn > 0 ? rn / fn : 0.0;
}

template <typename T>
pd_status paradiag_impl(pd_ctx *c, double *u, const double *f, const double *u0, int *h_iters,
                        double *h_relres, double *stats) {
  Prec<T> &P = prec<T>(c);
  LevelBufs &B = P.lv[0];
  const int N = c->N, n = c->n;
  const double h2 = hl(c, 0) * hl(c, 0);
  const View g = view(B.b, N, B.P);
  const View z0 = view(B.z[0], N, B.P), z1 = view(B.z[1], N, B.P);
  std::vector<int> it_sum(n, 0);
  int cyc_max_sum = 0;
  double st_local[PD_STATS_LEN];
  for (int k = 0; k < PD_STATS_LEN; k++) st_local[k] = 0.0;
  st_local[PD_STAT_RELRES_ALLATONCE] = -1.0;
  pd_status rc = PD_OK;
  const bool imag = c->cfg.imag_check != 0;
  c->outer_hist.clear();
  auto accumulate_iters = [&]() {
    int mx = 0;
    for (int j = 0; j < n; j++) {
      it_sum[j] += c->h_iters[j];
      mx = std::max(mx, c->h_iters[j]);
    }
    cyc_max_sum += mx;
  };
  if (imag) ck(c, cudaMemsetAsync(c->d_imag, 0, sizeof(unsigned long long), c->stream));
  const double w = sizeof(typename Cx<T>::type), m = (double)N * N;
  const double fwd_bytes = (8.0 + w) * m, fwd_u0 = 8.0 * m / n;
  if (c->cfg.precision == 0) {
    PD_PROF(PD_KC_FORWARD, fwd_bytes + (u0 ? fwd_u0 : 0.0), 0,
            transform_forward<T>(c, g, f, u0, true));
    ck_launch(c);
    rc = solve_levels<T>(c, c->cfg.tol, c->cfg.maxit);
    accumulate_iters();
    PD_PROF(PD_KC_INVERSE, (w + 8.0) * m, 0,
            transform_inverse<T>(c, u, z0, z1, c->st.final_buf, false, imag));
    ck_launch(c);
    if (c->have_B) {
      const int outer = c->cfg.outer_maxit;
      double rn, fn;
      allatonce_norms(c, outer > 0 ? c->d_r : nullptr, u, f, u0, &rn, &fn);
      double relres = rel_of(rn, fn);
      c->outer_hist.push_back(relres);
      int steps = 1;
      // FP64 corrections: d = (V kron I)(D kron I + kappa I kron A)^{-1}(V^{-1} kron I) r
      for (int s = 0; s < outer && rc == PD_OK && relres > c->cfg.tol; s++) {
        PD_PROF(PD_KC_FORWARD, fwd_bytes, 0, transform_forward<T>(c, g, c->d_r, nullptr, true));
        ck_launch(c);
        rc = solve_levels<T>(c, c->cfg.tol, c->cfg.maxit);
        if (rc == PD_ERR_NAN) break;
        if (rc == PD_ERR_NOCONV) rc = PD_OK;  // the outer residual decides
        accumulate_iters();
        PD_PROF(PD_KC_INVERSE, (w + 16.0) * m, 0,
                transform_inverse<T>(c, u, z0, z1, c->st.final_buf, true, imag));
        ck_launch(c);
        allatonce_norms(c, c->d_r, u, f, u0, &rn, &fn);
        const double prev = relres;
        relres = rel_of(rn, fn);
        c->outer_hist.push_back(relres);
        steps++;
        if (!std::isfinite(relres)) {
          rc = PD_ERR_NAN;
          break;
        }
        if (relres > 0.9 * prev) break;  // no longer contracts
      }
      if (rc == PD_OK && !std::isfinite(relres)) rc = PD_ERR_NAN;
      st_local[PD_STAT_RELRES_ALLATONCE] = relres;
      st_local[PD_STAT_REFINE_STEPS] = outer > 0 ? steps : 0;
      if (outer > 0 && rc == PD_OK && !(relres <= c->cfg.tol)) rc = PD_ERR_NOCONV;
    }
  } else {
    // FP64 iterative refinement on eq. (1) around FP32 ParaDIAG steps.  Step 1 transforms
    // fhat itself; later steps transform the FP64 residual r = fhat - A u, handed to the
    // FP32 solve times a power of two 2^sig that keeps it near unit size whatever the
    // scale of the data (the FP32 norms inside the multigrid neither underflow nor
    // overflow), the correction added times 2^-sig.
    double relres = 1.0, prev_relres = 1.0;
    int steps = 0, sig = 0;
    for (int step = 0; step < std::max(1, c->cfg.max_refine); step++) {
      if (step == 0)
        PD_PROF(PD_KC_FORWARD, fwd_bytes + (u0 ? fwd_u0 : 0.0), 0,
                transform_forward<T>(c, g, f, u0, true));
      else if (c->bidiag)
        PD_PROF(PD_KC_FORWARD, fwd_bytes - 4.0 * m, 0,
                transform_forward<T>(c, g, c->d_r32, nullptr, true, true));
      else
        PD_PROF(PD_KC_FORWARD, fwd_bytes, 0,
                transform_forward<T>(c, g, c->d_r, nullptr, true, false, std::ldexp(1.0, sig)));
      ck_launch(c);
      pd_status s = solve_levels<T>(c, c->cfg.inner_tol, c->cfg.inner_maxit, c->cfg.stall_ratio, true);
      if (s == PD_ERR_NAN) {
        rc = s;
        break;
      }
      accumulate_iters();
      PD_PROF(PD_KC_INVERSE, (w + (step > 0 ? 16.0 : 8.0)) * m, 0,
              transform_inverse<T>(c, u, z0, z1, c->st.final_buf, step > 0, imag, std::ldexp(1.0, -sig)));
      ck_launch(c);
      double rn, fn;
      if (c->bidiag) {
        // predicted scale of the next residual: a refinement step reduces it about 20-fold
        sig += 4;
        allatonce_norms(c, nullptr, u, f, u0, &rn, &fn, c->d_r32, step == 0 ? -1.0 : c->fnorm,
                        step == 0 ? 1 : 2, &sig);
        c->fnorm = fn;
      } else {
        allatonce_norms(c, c->d_r, u, f, u0, &rn, &fn);
        const double rms = rn / std::sqrt(m * n);
        sig = rms > 0.0 && std::isfinite(rms)
                  ? std::max(-120, std::min(120, -(int)std::lround(std::log2(rms))))
                  : 0;
      }
      steps = step + 1;
      relres = rel_of(rn, fn);
      c->outer_hist.push_back(relres);
      if (!std::isfinite(relres)) {
        rc = PD_ERR_NAN;
        break;
      }
      if (relres <= c->cfg.tol) break;
      if (step >= 2 && relres > 0.9 * prev_relres) break;  // refinement no longer contracts
      prev_relres = relres;
    }
    st_local[PD_STAT_RELRES_ALLATONCE] = relres;
    st_local[PD_STAT_REFINE_STEPS] = steps;
    if (rc == PD_OK && !(relres <= c->cfg.tol)) rc = PD_ERR_NOCONV;
  }
  check_wait_flags(c);
  if (imag && P.tc && n > 64) {
    st_local[PD_STAT_IMAG_MAX] = -1.0;  // the tensor-core inverse for n > 64 forms Re only
  } else if (imag) {
    unsigned long long bits = 0;
    ck(c, cudaMemcpy(&bits, c->d_imag, sizeof(bits), cudaMemcpyDeviceToHost));
    double v;
    std::memcpy(&v, &bits, sizeof(v));
    st_local[PD_STAT_IMAG_MAX] = v;
  }
  double tot = 0.0, rmax = 0.0;
  for (int j = 0; j < n; j++) {
    tot += it_sum[j];
    rmax = std::max(rmax, c->h_relres[j]);
    if (h_iters) h_iters[j] = it_sum[j];
    if (h_relres) h_relres[j] = c->h_relres[j];
  }
  st_local[PD_STAT_CYCLES_TOTAL] = tot;
  st_local[PD_STAT_CYCLES_MAX] = cyc_max_sum;
  st_local[PD_STAT_RELRES_SHIFT_MAX] = rmax;
  if (stats)
    for (int k = 0; k < PD_STATS_LEN; k++) stats[k] = st_local[k];
  return rc;
}

bool is_pow2m1(int N) { return N >= 1 && ((N + 1) & N) == 0; }

#define PD_TRY(ctx, ...)                    \
  try {                                     \
    __VA_ARGS__                             \
  } catch (const CudaFail &) {              \
    return PD_ERR_CUDA;                     \
  } catch (const std::bad_alloc &) {        \
    return PD_ERR_NOMEM;                    \
  } catch (pd_status s_) {                  \
    return s_;                              \
  }

void free_ctx(pd_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void *p : c->allocs) cudaFree(p);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->h_iters) cudaFreeHost(c->h_iters);
  if (c->h_relres) cudaFreeHost(c->h_relres);
  if (c->h_part) cudaFreeHost(c->h_part);
  if (c->h_hist) cudaFreeHost(c->h_hist);
  if (c->h_frozen) cudaFreeHost(c->h_frozen);
  if (c->h_srpart) cudaFreeHost(c->h_srpart);
  if (c->h_rsc) cudaFreeHost(c->h_rsc);
  for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  for (int k = 0; k < 2; k++)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  if (c->copy_stream_out) {
    cudaStreamSynchronize(c->copy_stream_out);
    cudaStreamDestroy(c->copy_stream_out);
  }
  for (int q = 0; q < 2; q++) {
    if (c->ev_in[q]) cudaEventDestroy(c->ev_in[q]);
    if (c->ev_done[q]) cudaEventDestroy(c->ev_done[q]);
    if (c->ev_out[q]) cudaEventDestroy(c->ev_out[q]);
  }
  delete c;
}

}  // namespace

extern "C" {

void pd_config_default(pd_config *cfg) {
  if (!cfg) return;
  cfg->cycle_gamma = 1;
  cfg->nu1 = 1;
  cfg->nu2 = 1;
  cfg->coarsest_n = 3;
  cfg->maxit = 100;
  cfg->tol = 1e-10;
  cfg->omega_mode = 1;
  cfg->precision = 0;
  cfg->smoother = 0;
  cfg->inner_tol = 1e-6;
  cfg->max_refine = 12;
  cfg->imag_check = 1;
  cfg->inner_maxit = 2;
  cfg->stall_ratio = 0.5;
  cfg->fused = 1;
  cfg->tensor_transforms = 1;
  cfg->fused_variant = 0;
  cfg->kappa = 1.0;
  cfg->outer_maxit = 0;
  cfg->cuda_graphs = 1;
  cfg->fx_residual = 1;
  cfg->fft_transforms = 1;
}

pd_status pd_diagonalize(int n, const double *B, double *shifts, double *V, double *Vinv) {
  if (n < 1 || n > 4096 || !B) return PD_ERR_ARG;
  std::vector<double> lam, v, vi;
  try {
    if (diagonalize(n, B, lam, v, vi) != 0) return PD_ERR_SING;
  } catch (const std::bad_alloc &) {
    return PD_ERR_NOMEM;
  }
  if (shifts) std::memcpy(shifts, lam.data(), lam.size() * sizeof(double));
  if (V) std::memcpy(V, v.data(), v.size() * sizeof(double));
  if (Vinv) std::memcpy(Vinv, vi.data(), vi.size() * sizeof(double));
  return PD_OK;
}

pd_status pd_shifts_alpha_circulant(int n, double tau, double alpha, double *shifts, double *V,
                                    double *Vinv) {
  return pd_alpha_circulant(n, tau, alpha, nullptr, shifts, V, Vinv, nullptr);
}

pd_status pd_alpha_circulant(int n, double tau, double alpha, double *B, double *shifts,
                             double *V, double *Vinv, double *u0coef) {
  if (n < 1 || !(tau > 0) || !(alpha > 0) || alpha > 1) return PD_ERR_ARG;
  const double an = std::pow(alpha, 1.0 / n);
  for (int j = 0; j < n; j++) {
    const std::complex<double> e = std::polar(1.0, 2.0 * M_PI * j / n);
    const std::complex<double> lam = (1.0 - an * e) / tau;
    if (shifts) {
      shifts[2 * j] = lam.real();
      shifts[2 * j + 1] = lam.imag();
    }
  }
  for (int k = 0; k < n; k++)
    for (int j = 0; j < n; j++) {
      const size_t e = (size_t)k * n + j;
      const double ang = 2.0 * M_PI * (double)((long long)k * j % n) / n;
      if (V) {
        const std::complex<double> v = std::pow(alpha, -(double)k / n) * std::polar(1.0, -ang);
        V[2 * e] = v.real();
        V[2 * e + 1] = v.imag();
      }
      if (Vinv) {
        const std::complex<double> v = std::polar(1.0, ang) * std::pow(alpha, (double)j / n) / (double)n;
        Vinv[2 * e] = v.real();
        Vinv[2 * e + 1] = v.imag();
      }
      if (B) {
        double b = 0.0;
        if (k == j) b = 1.0 / tau;
        if (k == j + 1) b = -1.0 / tau;
        if (k == 0 && j == n - 1) b += -alpha / tau;
        B[e] = b;
      }
    }
  if (u0coef)
    for (int k = 0; k < n; k++) u0coef[k] = (k == 0) ? 1.0 / tau : 0.0;
  return PD_OK;
}

pd_status paradiag_setup(pd_ctx **out, int N, double h, int n, const double *shifts,
                         const double *V, const double *Vinv, const double *B,
                         const double *u0coef, const double *omega, const pd_config *cfg_in,
                         void *stream) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  pd_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else pd_config_default(&cfg);
  if (!is_pow2m1(N) || n < 1 || n > kMaxShifts) return PD_ERR_ARG;
  // B alone: the library diagonalises it (B = V D V^{-1}, Sec. 1)
  std::vector<double> eig_lam, eig_V, eig_Vinv;
  if (!shifts) {
    if (!B || V || Vinv) return PD_ERR_ARG;
    if (diagonalize(n, B, eig_lam, eig_V, eig_Vinv) != 0) return PD_ERR_SING;
    shifts = eig_lam.data();
    V = eig_V.data();
    Vinv = eig_Vinv.data();
  }
  if (!(std::fabs(h * (N + 1) - 1.0) <= 1e-12)) return PD_ERR_ARG;
  if ((V == nullptr) != (Vinv == nullptr)) return PD_ERR_ARG;
  if (!(cfg.coarsest_n == 1 || cfg.coarsest_n == 3 || cfg.coarsest_n == 7 || cfg.coarsest_n == 15))
    return PD_ERR_ARG;
  if (N < cfg.coarsest_n || cfg.cycle_gamma < 1 || cfg.cycle_gamma > 2 || cfg.nu1 < 0 ||
      cfg.nu2 < 0 || cfg.nu1 + cfg.nu2 < 1 || cfg.nu1 > 8 || cfg.nu2 > 8 || cfg.maxit < 0 ||
      cfg.maxit > 100000 || !(cfg.tol >= 0) || cfg.omega_mode < 0 || cfg.omega_mode > 2 ||
      cfg.precision < 0 || cfg.precision > 1 || cfg.smoother < 0 || cfg.smoother > 1 ||
      !(cfg.inner_tol >= 0) || cfg.max_refine < 1 || cfg.inner_maxit < 1 ||
      cfg.inner_maxit > 100000 || !(cfg.stall_ratio >= 0) || cfg.fused < 0 || cfg.fused > 2 ||
      cfg.tensor_transforms < 0 || cfg.tensor_transforms > 1 || cfg.fused_variant < 0 ||
      cfg.fused_variant > 2 || !(cfg.kappa > 0) || !std::isfinite(cfg.kappa) ||
      cfg.outer_maxit < 0 || cfg.outer_maxit > 1000 || cfg.cuda_graphs < 0 || cfg.cuda_graphs > 1 ||
      cfg.fx_residual < 0 || cfg.fx_residual > 1 || cfg.fft_transforms < 0 ||
      cfg.fft_transforms > 1)
    return PD_ERR_ARG;
  if (cfg.precision == 0 && cfg.outer_maxit > 0 && (!B || !V)) return PD_ERR_ARG;
  if (cfg.omega_mode == 2 && !omega) return PD_ERR_ARG;
  // precision 1 needs B (the refinement residual of eq. (1)) with V, or neither (shifted
  // solves only)
  if (cfg.precision == 1 && (B == nullptr) != (V == nullptr)) return PD_ERR_ARG;
  for (int k = 0; k < 2 * n; k++)
    if (!std::isfinite(shifts[k])) return PD_ERR_ARG;
  pd_ctx *c = new (std::nothrow) pd_ctx();
  if (!c) return PD_ERR_NOMEM;
  c->N = N;
  c->n = n;
  c->cfg = cfg;
  c->kappa = cfg.kappa;
  int Nl = N;
  c->Ns.push_back(Nl);
  while (Nl > cfg.coarsest_n) {
    Nl = (Nl - 1) / 2;
    c->Ns.push_back(Nl);
  }
  c->L = (int)c->Ns.size();
  if (c->L > kMaxLevels) {
    delete c;
    return PD_ERR_ARG;
  }
  c->shifts.assign(shifts, shifts + 2 * n);
  c->have_V = V != nullptr;
  if (V) {
    c->V.assign(V, V + 2 * (size_t)n * n);
    c->Vinv.assign(Vinv, Vinv + 2 * (size_t)n * n);
  }
  c->have_B = B != nullptr;
  if (B) c->B.assign(B, B + (size_t)n * n);
  c->u0coef.assign(n, 0.0);
  if (u0coef) c->u0coef.assign(u0coef, u0coef + n);
  // relaxation parameters per shift and level
  c->omega.assign((size_t)n * c->L, 0.0);
  for (int j = 0; j < n; j++)
    for (int l = 0; l < c->L; l++) {
      double w;
      if (cfg.omega_mode == 2) w = omega[(size_t)j * c->L + l];
      else if (cfg.omega_mode == 0) w = cfg.smoother == 1 ? 0.8 : 24.0 / 25.0;
      else {
        const double hh = 1.0 / (c->Ns[l] + 1);
        w = lfa_omega_opt(shifts[2 * j] * hh * hh / cfg.kappa, shifts[2 * j + 1] * hh * hh / cfg.kappa,
                          cfg.smoother);
      }
      c->omega[(size_t)j * c->L + l] = w;
    }
  // plan of the coarse levels run inside one CTA per shift
  c->plan.L = c->L;
  for (int l = 0; l < c->L; l++) c->plan.Ns[l] = c->Ns[l];
  c->plan.gamma = cfg.cycle_gamma;
  c->plan.nu1 = cfg.nu1;
  c->plan.nu2 = cfg.nu2;
  c->plan.jacobi = cfg.smoother == 1;
  const int cap = cfg.precision == 0 ? 31 : 63;
  c->lc = c->L - 1;
  for (int l = c->L - 1; l >= 0; l--) {
    const size_t bytes = cfg.precision == 0 ? coarse_smem_bytes<double>(c->plan, l)
                                            : coarse_smem_bytes<float>(c->plan, l);
    if (bytes <= kCoarseSmemLimit && c->Ns[l] <= cap && c->L - 1 - l <= kMaxCoarseDepth) c->lc = l;
    else break;
  }
  c->plan.lc = c->lc;
  try {
    c->stream = (cudaStream_t)stream;
    for (int k = 0; k < 2; k++) ck(c, cudaEventCreateWithFlags(&c->ev[k], cudaEventDisableTiming));
    ck(c, cudaMallocHost(&c->h_pinned, 4 * sizeof(int)));
    ck(c, cudaMallocHost(&c->h_iters, n * sizeof(int)));
    ck(c, cudaMallocHost(&c->h_relres, n * sizeof(double)));
    {
      int dev = 0;
      ck(c, cudaGetDevice(&dev));
      ck(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    ck(c, cudaMallocHost(&c->h_part, 2 * part_blocks(c) * sizeof(double)));
    ck(c, cudaMallocHost(&c->h_hist, (std::max(cfg.maxit, cfg.inner_maxit) + 2) * sizeof(int)));
    {
      const int gx = shift_residual_blocks(N, n, c->num_sms);
      ck(c, cudaMallocHost(&c->h_frozen, n * sizeof(int)));
      ck(c, cudaMallocHost(&c->h_rsc, n * sizeof(float)));
      c->d_rsc = dalloc<float *>(c, n * sizeof(float));
      ck(c, cudaMallocHost(&c->h_srpart, 2 * (size_t)n * gx * sizeof(double)));
      c->d_frozen = dalloc<int *>(c, n * sizeof(int));
      c->d_srpart = dalloc<double *>(c, 2 * (size_t)n * gx * sizeof(double));
      c->d_c1 = dalloc<double2 *>(c, n * sizeof(double2));
      std::vector<double2> c1(n);
      const double hh = 1.0 / (N + 1);
      for (int j = 0; j < n; j++)
        c1[j] = make_double2(shifts[2 * j] + 4.0 * cfg.kappa / (hh * hh), shifts[2 * j + 1]);
      ck(c, cudaMemcpy(c->d_c1, c1.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
      c->d_lam = dalloc<double2 *>(c, n * sizeof(double2));
      ck(c, cudaMemcpy(c->d_lam, shifts, n * sizeof(double2), cudaMemcpyHostToDevice));
      ck(c, cudaMemset(c->d_frozen, 0, n * sizeof(int)));
    }
    // solve state
    const FusedGeom g32 = fused_geom<float>(), g64 = fused_geom<double>();
    const int tiles = std::max({smooth_tiles(N), fused_tiles(N, g32.TX, g32.TY),
                                fused_tiles(N, g64.TX, g64.TY), stream_units(N, 4)});
    c->st.max_tiles = tiles;
    c->st.active = dalloc<int *>(c, n * sizeof(int));
    c->st.iters = dalloc<int *>(c, n * sizeof(int));
    c->st.final_buf = dalloc<int *>(c, n * sizeof(int));
    c->st.nactive = dalloc<int *>(c, 2 * sizeof(int));
    c->st.flags = c->st.nactive + 1;
    // the wait flags are read after standalone component calls that never reset the state
    ck(c, cudaMemset(c->st.nactive, 0, 2 * sizeof(int)));
    c->st.bn2 = dalloc<double *>(c, n * sizeof(double));
    c->st.relres = dalloc<double *>(c, n * sizeof(double));
    c->st.partials = dalloc<double *>(c, (size_t)n * tiles * sizeof(double));
    c->st.hist_stride = std::max(cfg.maxit, cfg.inner_maxit) + 1;
    c->st.hist = dalloc<double *>(c, (size_t)n * c->st.hist_stride * sizeof(double));
    c->d_u0coef = dalloc<double *>(c, n * sizeof(double));
    ck(c, cudaMemcpy(c->d_u0coef, c->u0coef.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    c->d_part = dalloc<double *>(c, 2 * part_blocks(c) * sizeof(double));
    c->d_imag = dalloc<unsigned long long *>(c, sizeof(unsigned long long));
    ck(c, cudaMemset(c->d_imag, 0, sizeof(unsigned long long)));
    if (B) {
      std::vector<double> bd(n), bs(n);
      for (int off = -1; off <= 1 && !c->bidiag; off += 2) {
        bool bid = n > 1;
        for (int k = 0; k < n; k++) {
          const int kp = (k + off + n) % n;
          bd[k] = B[(size_t)k * n + k];
          bs[k] = n > 1 ? B[(size_t)k * n + kp] : 0.0;
          for (int l = 0; l < n; l++)
            if (B[(size_t)k * n + l] != 0.0 && l != k && l != kp) bid = false;
        }
        if (bid && n > 2) {
          c->bidiag = true;
          c->boff = off;
        }
      }
      if (c->bidiag) {
        c->d_bd = dalloc<double *>(c, n * sizeof(double));
        c->d_bs = dalloc<double *>(c, n * sizeof(double));
        ck(c, cudaMemcpy(c->d_bd, bd.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        ck(c, cudaMemcpy(c->d_bs, bs.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        // the same constants as float-float pairs for the FP64-free residual
        std::vector<float4> kbd(n);
        std::vector<float2> ku0(n);
        for (int k = 0; k < n; k++) {
          const float2 a = split_ff(bd[k]), b = split_ff(bs[k]);
          kbd[k] = make_float4(a.x, a.y, b.x, b.y);
          ku0[k] = split_ff(c->u0coef[k]);
        }
        const double hh = 1.0 / (N + 1);
        c->ihf = split_ff(cfg.kappa / (hh * hh));
        c->d_kbd = dalloc<float4 *>(c, n * sizeof(float4));
        c->d_ku0 = dalloc<float2 *>(c, n * sizeof(float2));
        ck(c, cudaMemcpy(c->d_kbd, kbd.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
        ck(c, cudaMemcpy(c->d_ku0, ku0.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
      }
      std::vector<int> ptr(n + 1, 0), col;
      std::vector<double> val;
      for (int k = 0; k < n; k++) {
        for (int l = 0; l < n; l++)
          if (B[(size_t)k * n + l] != 0.0) {
            col.push_back(l);
            val.push_back(B[(size_t)k * n + l]);
          }
        ptr[k + 1] = (int)col.size();
      }
      c->d_Bptr = dalloc<int *>(c, ptr.size() * sizeof(int));
      c->d_Bcol = dalloc<int *>(c, std::max<size_t>(col.size(), 1) * sizeof(int));
      c->d_Bval = dalloc<double *>(c, std::max<size_t>(val.size(), 1) * sizeof(double));
      ck(c, cudaMemcpy(c->d_Bptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
      if (!col.empty()) {
        ck(c, cudaMemcpy(c->d_Bcol, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice));
        ck(c, cudaMemcpy(c->d_Bval, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice));
      }
    }
    if (cfg.precision == 0) {
      alloc_prec<double>(c);
      if (cfg.outer_maxit > 0) c->d_r = dalloc<double *>(c, (size_t)n * N * N * sizeof(double));
    } else {
      alloc_prec<float>(c);
      if (c->have_B) {
        if (c->bidiag) c->d_r32 = dalloc<float *>(c, (size_t)n * N * N * sizeof(float));
        if (c->bidiag && cfg.fx_residual)
          c->d_fcache = dalloc<float2 *>(c, (size_t)n * N * N * sizeof(float2));
        else c->d_r = dalloc<double *>(c, (size_t)n * N * N * sizeof(double));
      }
    }
    ck(c, cudaDeviceSynchronize());
  } catch (const CudaFail &) {
    free_ctx(c);
    return PD_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    free_ctx(c);
    return PD_ERR_NOMEM;
  } catch (pd_status s) {
    free_ctx(c);
    return s;
  }
  *out = c;
  return PD_OK;
}

pd_status pd_adjoint_setup(const pd_ctx *c, pd_ctx **out) {
  if (!c || !out) return PD_ERR_ARG;
  if (!c->have_V) return PD_ERR_STATE;
  const int n = c->n;
  std::vector<double> sh(2 * n), Va(2 * (size_t)n * n), Via(2 * (size_t)n * n), Bt;
  for (int j = 0; j < n; j++) {
    sh[2 * j] = c->shifts[2 * j];
    sh[2 * j + 1] = -c->shifts[2 * j + 1];
  }
  // V_adj = (V^{-1})^H, V_adj^{-1} = V^H
  for (int k = 0; k < n; k++)
    for (int j = 0; j < n; j++) {
      const size_t e = (size_t)k * n + j, t = (size_t)j * n + k;
      Va[2 * e] = c->Vinv[2 * t];
      Va[2 * e + 1] = -c->Vinv[2 * t + 1];
      Via[2 * e] = c->V[2 * t];
      Via[2 * e + 1] = -c->V[2 * t + 1];
    }
  if (c->have_B) {
    Bt.resize((size_t)n * n);
    for (int k = 0; k < n; k++)
      for (int l = 0; l < n; l++) Bt[(size_t)k * n + l] = c->B[(size_t)l * n + k];
  }
  pd_config cfg = c->cfg;
  cfg.omega_mode = 2;  // conj(lam) has the same LFA optimum; reuse the forward table
  return paradiag_setup(out, c->N, 1.0 / (c->N + 1), n, sh.data(), Va.data(), Via.data(),
                        c->have_B ? Bt.data() : nullptr, nullptr, c->omega.data(), &cfg, c->stream);
}

int pd_num_levels(const pd_ctx *c) { return c ? c->L : 0; }

pd_status pd_get_omega(const pd_ctx *c, double *h_omega) {
  if (!c || !h_omega) return PD_ERR_ARG;
  std::memcpy(h_omega, c->omega.data(), c->omega.size() * sizeof(double));
  return PD_OK;
}

pd_status mg_vcycle(pd_ctx *c, int level, void *z, const void *b) {
  if (!c || !z || !b || level < 0 || level >= c->L) return PD_ERR_ARG;
  PD_TRY(c, {
    const int N = c->Ns[level], n = c->n;
    const double h = hl(c, level);
    if (c->cfg.precision == 0) {
      LevelBufs &B = c->p64.lv[level];
      launch_copy_scale<double>(c->stream, N, n, view(B.b, N, B.P), uview(b, N), rs(c, level));
      launch_copy_scale<double>(c->stream, N, n, view(B.z[0], N, B.P), uview(z, N), 1.0);
      ck_launch(c, 2);
      c->cur[level] = 0;
      run_cycle<double>(c, level, false, false, nullptr, 0.0, 0);
      launch_copy_scale<double>(c->stream, N, n, uview(z, N), view(B.z[c->cur[level]], N, B.P), 1.0);
    } else {
      LevelBufs &B = c->p32.lv[level];
      launch_copy_scale<float>(c->stream, N, n, view(B.b, N, B.P), uview(b, N), (float)rs(c, level));
      launch_copy_scale<float>(c->stream, N, n, view(B.z[0], N, B.P), uview(z, N), 1.0f);
      ck_launch(c, 2);
      c->cur[level] = 0;
      run_cycle<float>(c, level, false, false, nullptr, 0.0, 0);
      launch_copy_scale<float>(c->stream, N, n, uview(z, N), view(B.z[c->cur[level]], N, B.P), 1.0f);
    }
    ck_launch(c);
    return PD_OK;
  })
}

pd_status shifted_solve_batched(pd_ctx *c, void *z, const void *b, int *h_iters, double *h_relres) {
  if (!c || !z || !b) return PD_ERR_ARG;
  PD_TRY(c, {
    const int N = c->N, n = c->n;
    const double h = hl(c, 0);
    pd_status rc;
    if (c->cfg.precision == 0) {
      LevelBufs &B = c->p64.lv[0];
      launch_copy_scale<double>(c->stream, N, n, view(B.b, N, B.P), uview(b, N), rs(c, 0));
      ck_launch(c);
      rc = solve_levels<double>(c, c->cfg.tol, c->cfg.maxit);
      launch_gather_final<double>(c->stream, N, n, uview(z, N), view(B.z[0], N, B.P),
                                  view(B.z[1], N, B.P), c->st.final_buf);
    } else {
      LevelBufs &B = c->p32.lv[0];
      launch_copy_scale<float>(c->stream, N, n, view(B.b, N, B.P), uview(b, N), (float)rs(c, 0));
      ck_launch(c);
      rc = solve_levels<float>(c, c->cfg.tol, c->cfg.maxit);
      launch_gather_final<float>(c->stream, N, n, uview(z, N), view(B.z[0], N, B.P),
                                 view(B.z[1], N, B.P), c->st.final_buf);
    }
    ck_launch(c);
    ck(c, cudaStreamSynchronize(c->stream));
    for (int j = 0; j < n; j++) {
      if (h_iters) h_iters[j] = c->h_iters[j];
      if (h_relres) h_relres[j] = c->h_relres[j];
    }
    return rc;
  })
}

pd_status paradiag_solve(pd_ctx *c, double *u, const double *f, const double *u0, int *h_iters,
                         double *h_relres, double *h_stats) {
  if (!c || !u || !f) return PD_ERR_ARG;
  if (!c->have_V) return PD_ERR_STATE;
  PD_TRY(c, {
    if (c->cfg.precision == 0) return paradiag_impl<double>(c, u, f, u0, h_iters, h_relres, h_stats);
    return paradiag_impl<float>(c, u, f, u0, h_iters, h_relres, h_stats);
  })
}

pd_status paradiag_solve_host(pd_ctx *c, double *h_u, const double *h_f, const double *h_u0,
                              int *h_iters, double *h_relres, double *h_stats) {
  if (!c || !h_u || !h_f) return PD_ERR_ARG;
  if (!c->have_V) return PD_ERR_STATE;
  PD_TRY(c, {
    const size_t bytes = (size_t)c->n * c->N * c->N * sizeof(double);
    const size_t b0 = (size_t)c->N * c->N * sizeof(double);
    if (!c->d_stage_f) {
      c->d_stage_f = dalloc<double *>(c, bytes);
      c->d_stage_u = dalloc<double *>(c, bytes);
      c->d_stage_u0 = dalloc<double *>(c, b0);
    }
    ck(c, cudaMemcpyAsync(c->d_stage_f, h_f, bytes, cudaMemcpyHostToDevice, c->stream));
    if (h_u0) ck(c, cudaMemcpyAsync(c->d_stage_u0, h_u0, b0, cudaMemcpyHostToDevice, c->stream));
    pd_status rc = paradiag_solve(c, c->d_stage_u, c->d_stage_f, h_u0 ? c->d_stage_u0 : nullptr,
                                  h_iters, h_relres, h_stats);
    if (rc == PD_ERR_CUDA) return rc;
    ck(c, cudaMemcpyAsync(h_u, c->d_stage_u, bytes, cudaMemcpyDeviceToHost, c->stream));
    ck(c, cudaStreamSynchronize(c->stream));
    return rc;
  })
}

namespace {
// the device address of page-locked (pinned or registered) host memory, or nullptr for
// pageable memory
void *host_device_pointer(void *h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // pageable memory on older runtimes reports an error: clear it
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
}  // namespace

pd_status paradiag_solve_host_batch(pd_ctx *c, int count, double *const *h_u,
                                    const double *const *h_f, const double *const *h_u0,
                                    int *h_iters, double *h_relres, double *h_stats) {
  if (!c || count < 1 || !h_u || !h_f) return PD_ERR_ARG;
  for (int k = 0; k < count; k++)
    if (!h_u[k] || !h_f[k]) return PD_ERR_ARG;
  if (!c->have_V) return PD_ERR_STATE;
  PD_TRY(c, {
    const size_t bytes = (size_t)c->n * c->N * c->N * sizeof(double);
    const size_t b0 = (size_t)c->N * c->N * sizeof(double);
    if (!c->copy_stream) {
      ck(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
      ck(c, cudaStreamCreateWithFlags(&c->copy_stream_out, cudaStreamNonBlocking));
      for (int q = 0; q < 2; q++) {
        c->d_pf[q] = dalloc<double *>(c, bytes);
        c->d_pu[q] = dalloc<double *>(c, bytes);
        c->d_pu0[q] = dalloc<double *>(c, b0);
        ck(c, cudaEventCreateWithFlags(&c->ev_in[q], cudaEventDisableTiming));
        ck(c, cudaEventCreateWithFlags(&c->ev_done[q], cudaEventDisableTiming));
        ck(c, cudaEventCreateWithFlags(&c->ev_out[q], cudaEventDisableTiming));
      }
    }
    // the copy streams start after the work queued on the context's stream before the call
    ck(c, cudaEventRecord(c->ev_done[1], c->stream));
    ck(c, cudaStreamWaitEvent(c->copy_stream, c->ev_done[1], 0));
    ck(c, cudaStreamWaitEvent(c->copy_stream_out, c->ev_done[1], 0));
    auto copy_in = [&](int j) {
      const int q = j & 1;
      if (j >= 2) ck(c, cudaStreamWaitEvent(c->copy_stream, c->ev_done[q], 0));  // solve j-2 done
      ck(c, cudaMemcpyAsync(c->d_pf[q], h_f[j], bytes, cudaMemcpyHostToDevice, c->copy_stream));
      if (h_u0 && h_u0[j])
        ck(c, cudaMemcpyAsync(c->d_pu0[q], h_u0[j], b0, cudaMemcpyHostToDevice, c->copy_stream));
      ck(c, cudaEventRecord(c->ev_in[q], c->copy_stream));
    };
    copy_in(0);
    pd_status worst = PD_OK;
    for (int k = 0; k < count; k++) {
      const int q = k & 1;
      if (k + 1 < count) copy_in(k + 1);
      ck(c, cudaStreamWaitEvent(c->stream, c->ev_in[q], 0));
      if (k >= 2) ck(c, cudaStreamWaitEvent(c->stream, c->ev_out[q], 0));  // u of k-2 copied out
      const pd_status rc = paradiag_solve(c, c->d_pu[q], c->d_pf[q],
                                          (h_u0 && h_u0[k]) ? c->d_pu0[q] : nullptr,
                                          h_iters ? h_iters + (size_t)k * c->n : nullptr,
                                          h_relres ? h_relres + (size_t)k * c->n : nullptr,
                                          h_stats ? h_stats + (size_t)k * PD_STATS_LEN : nullptr);
      if (rc == PD_ERR_CUDA) return rc;
      if (worst == PD_OK && rc != PD_OK) worst = rc;
      ck(c, cudaEventRecord(c->ev_done[q], c->stream));
      ck(c, cudaStreamWaitEvent(c->copy_stream_out, c->ev_done[q], 0));
      // u out: into mapped pinned memory by a streaming copy kernel on 32 CTAs (beside the
      // next solve it slows that solve less than a copy-engine transfer: 170 against 177 ms
      // at 2047^2 x 128, measured), else by the copy engine
      void *dptr = host_device_pointer(h_u[k]);
      if (dptr && bytes % 16 == 0 && reinterpret_cast<uintptr_t>(dptr) % 16 == 0) {
        launch_stream_copy(c->copy_stream_out, 32, c->d_pu[q], dptr, (long long)(bytes / 16));
        ck_launch(c);
      } else {
        ck(c, cudaMemcpyAsync(h_u[k], c->d_pu[q], bytes, cudaMemcpyDeviceToHost, c->copy_stream_out));
      }
      ck(c, cudaEventRecord(c->ev_out[q], c->copy_stream_out));
    }
    ck(c, cudaStreamSynchronize(c->copy_stream));
    ck(c, cudaStreamSynchronize(c->copy_stream_out));
    return worst;
  })
}

pd_status pd_smooth(pd_ctx *c, int level, void *zout, const void *zin, const void *b) {
  if (!c || !zout || !zin || !b || zout == zin || level < 0 || level >= c->L) return PD_ERR_ARG;
  PD_TRY(c, {
    const int N = c->Ns[level], n = c->n;
    const double h = hl(c, level);
    const bool jac = c->cfg.smoother == 1;
    if (c->cfg.precision == 0)
      launch_smooth<double>(c->stream, N, n, uview(zin, N), uview(zout, N), uview(b, N), rs(c, level),
                            c->p64.coef + (size_t)level * n, nullptr, false, jac, nullptr, 0);
    else
      launch_smooth<float>(c->stream, N, n, uview(zin, N), uview(zout, N), uview(b, N),
                           (float)rs(c, level), c->p32.coef + (size_t)level * n, nullptr, false, jac,
                           nullptr, 0);
    ck_launch(c);
    return PD_OK;
  })
}

pd_status pd_residual_restrict(pd_ctx *c, int level, void *bc, const void *z, const void *b) {
  if (!c || !bc || !z || !b || level < 0 || level >= c->L - 1) return PD_ERR_ARG;
  PD_TRY(c, {
    const int N = c->Ns[level], Nc = c->Ns[level + 1], n = c->n;
    const double h = hl(c, level), hc = hl(c, level + 1);
    if (c->cfg.precision == 0)
      launch_residual_restrict<double>(c->stream, N, n, uview(z, N), uview(b, N), rs(c, level),
                                       uview(bc, Nc), c->kappa / (hc * hc),
                                       c->p64.coef + (size_t)level * n, nullptr, false);
    else
      launch_residual_restrict<float>(c->stream, N, n, uview(z, N), uview(b, N), (float)rs(c, level),
                                      uview(bc, Nc), (float)(c->kappa / (hc * hc)),
                                      c->p32.coef + (size_t)level * n, nullptr, false);
    ck_launch(c);
    return PD_OK;
  })
}

pd_status pd_prolong_add(pd_ctx *c, int level, void *z, const void *ec) {
  if (!c || !z || !ec || level < 0 || level >= c->L - 1) return PD_ERR_ARG;
  PD_TRY(c, {
    const int N = c->Ns[level], Nc = c->Ns[level + 1], n = c->n;
    if (c->cfg.precision == 0)
      launch_prolong_add<double>(c->stream, N, n, uview(z, N), uview(ec, Nc), nullptr);
    else
      launch_prolong_add<float>(c->stream, N, n, uview(z, N), uview(ec, Nc), nullptr);
    ck_launch(c);
    return PD_OK;
  })
}

pd_status pd_coarse_solve(pd_ctx *c, void *z, const void *b) {
  if (!c || !z || !b) return PD_ERR_ARG;
  PD_TRY(c, {
    const int l = c->L - 1, N = c->Ns[l], n = c->n;
    const double h = hl(c, l);
    if (c->cfg.precision == 0)
      launch_coarse<double>(c->stream, c->plan, l, n, uview(b, N), rs(c, l), uview(z, N), c->p64.coef,
                            c->p64.cinv, nullptr, 1, 0, 0, 0.0, 0, c->st);
    else
      launch_coarse<float>(c->stream, c->plan, l, n, uview(b, N), (float)rs(c, l), uview(z, N),
                           c->p32.coef, c->p32.cinv, nullptr, 1, 0, 0, 0.0, 0, c->st);
    ck_launch(c);
    return PD_OK;
  })
}

pd_status pd_transform_forward(pd_ctx *c, void *g, const double *f, const double *u0) {
  if (!c || !g || !f) return PD_ERR_ARG;
  if (!c->have_V) return PD_ERR_STATE;
  PD_TRY(c, {
    if (c->cfg.precision == 0)
      transform_forward<double>(c, uview(g, c->N), f, u0, false);
    else
      transform_forward<float>(c, uview(g, c->N), f, u0, false);
    ck_launch(c);
    check_wait_flags(c);
    return PD_OK;
  })
}

pd_status pd_transform_inverse(pd_ctx *c, double *u, const void *z, int accumulate) {
  if (!c || !u || !z) return PD_ERR_ARG;
  if (!c->have_V) return PD_ERR_STATE;
  PD_TRY(c, {
    const View zv = uview(z, c->N);
    if (c->cfg.precision == 0)
      transform_inverse<double>(c, u, zv, zv, nullptr, accumulate != 0, false);
    else
      transform_inverse<float>(c, u, zv, zv, nullptr, accumulate != 0, false);
    ck_launch(c);
    check_wait_flags(c);
    return PD_OK;
  })
}

pd_status pd_allatonce_residual(pd_ctx *c, double *r, const double *u, const double *f,
                                const double *u0, double *h_norms) {
  if (!c || !u || !f) return PD_ERR_ARG;
  if (!c->have_B) return PD_ERR_STATE;
  PD_TRY(c, {
    double rn, fn;
    allatonce_norms(c, r, u, f, u0, &rn, &fn);
    if (h_norms) {
      h_norms[0] = rn;
      h_norms[1] = fn;
    }
    return PD_OK;
  })
}

pd_status pd_laplacian_dot(pd_ctx *c, const double *w, const double *u, double *h_out) {
  if (!c || !w || !u || !h_out) return PD_ERR_ARG;
  PD_TRY(c, {
    PD_PROF(PD_KC_OTHER, 16.0 * c->N * c->N, 0,
            launch_laplacian_dot(c->stream, c->N, c->n, w, u, c->d_part));
    ck_launch(c);
    const int nb = allatonce_blocks();
    ck(c, cudaMemcpyAsync(c->h_part, c->d_part, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    ck(c, cudaStreamSynchronize(c->stream));
    double acc = 0.0;
    for (int k = 0; k < nb; k++) acc += c->h_part[2 * k];
    *h_out = acc;
    prof_resolve(c);
    return PD_OK;
  })
}

pd_status pd_initial_value_gradient(pd_ctx *c, const double *w, double *gu0) {
  if (!c || !w || !gu0) return PD_ERR_ARG;
  PD_TRY(c, {
    PD_PROF(PD_KC_OTHER, 16.0 * c->N * c->N, 0,
            launch_initial_value_gradient(c->stream, c->N, c->n, w, c->d_u0coef, gu0));
    ck_launch(c);
    return PD_OK;
  })
}

pd_status pd_profile_enable(pd_ctx *c, int on) {
  if (!c) return PD_ERR_ARG;
  PD_TRY(c, {
    ck(c, cudaStreamSynchronize(c->stream));
    prof_resolve(c);
    c->prof_on = on != 0;
    for (int k = 0; k < PD_KC_COUNT; k++) {
      c->prof_ms[k] = 0.0;
      c->prof_bytes[k] = 0.0;
      c->prof_n[k] = 0;
    }
    return PD_OK;
  })
}

pd_status pd_profile_read(pd_ctx *c, int kc, double *ms, long long *launches, double *bytes) {
  if (!c || kc < 0 || kc >= PD_KC_COUNT) return PD_ERR_ARG;
  PD_TRY(c, {
    ck(c, cudaStreamSynchronize(c->stream));
    prof_resolve(c);
    if (ms) *ms = c->prof_ms[kc];
    if (launches) *launches = c->prof_n[kc];
    if (bytes) *bytes = c->prof_bytes[kc];
    return PD_OK;
  })
}

pd_status pd_get_history(pd_ctx *c, int cap, int *h_cycle_len, double *h_cycle_hist, int cap_outer,
                         int *h_outer_len, double *h_outer) {
  if (!c || cap < 0 || cap_outer < 0) return PD_ERR_ARG;
  PD_TRY(c, {
    const int n = c->n, stride = c->st.hist_stride;
    ck(c, cudaStreamSynchronize(c->stream));
    std::vector<int> it(n);
    std::vector<double> h((size_t)n * stride);
    ck(c, cudaMemcpy(it.data(), c->st.iters, n * sizeof(int), cudaMemcpyDeviceToHost));
    ck(c, cudaMemcpy(h.data(), c->st.hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int j = 0; j < n; j++) {
      const int len = std::min(std::min(it[j] + 1, stride), cap);
      if (h_cycle_len) h_cycle_len[j] = len;
      if (h_cycle_hist)
        for (int k = 0; k < cap; k++) h_cycle_hist[(size_t)j * cap + k] = k < len ? h[(size_t)j * stride + k] : 0.0;
    }
    const int lo = std::min((int)c->outer_hist.size(), cap_outer);
    if (h_outer_len) *h_outer_len = lo;
    if (h_outer)
      for (int k = 0; k < cap_outer; k++) h_outer[k] = k < lo ? c->outer_hist[k] : 0.0;
    return PD_OK;
  })
}

pd_status pd_synchronize(pd_ctx *c) {
  if (!c) return PD_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->err = cudaGetErrorString(e);
    return PD_ERR_CUDA;
  }
  return PD_OK;
}

long long pd_launch_count(const pd_ctx *c) { return c ? c->launches : 0; }

pd_status pd_fused_choice(const pd_ctx *c, int level, int *h_variant, int *h_seg) {
  if (!c || level < 0 || level >= c->L) return PD_ERR_ARG;
  // the multigrid's working precision: FP32 levels in the precision form, FP64 otherwise
  const LevelBufs *B = nullptr;
  if (c->cfg.precision == 1 && level < (int)c->p32.lv.size()) B = &c->p32.lv[level];
  else if (c->cfg.precision == 0 && level < (int)c->p64.lv.size()) B = &c->p64.lv[level];
  // fused kernels run in FP32 with cfg.fused = 1 and in both precisions with cfg.fused = 2
  const bool on = c->cfg.fused == 2 || (c->cfg.fused == 1 && c->cfg.precision == 1);
  const bool fused = B && B->maps && level < c->L - 1 && on;
  if (h_variant) *h_variant = fused ? B->variant : 0;
  if (h_seg) *h_seg = fused && B->variant == 2 ? B->seg : 0;
  return PD_OK;
}

pd_status paradiag_destroy(pd_ctx *c) {
  if (!c) return PD_ERR_ARG;
  free_ctx(c);
  return PD_OK;
}

const char *pd_status_str(pd_status s) {
  switch (s) {
    case PD_OK: return "ok";
    case PD_ERR_ARG: return "invalid argument";
    case PD_ERR_CUDA: return "CUDA error";
    case PD_ERR_NOMEM: return "out of memory";
    case PD_ERR_NOCONV: return "tolerance not reached";
    case PD_ERR_NAN: return "NaN or Inf in a residual";
    case PD_ERR_SING: return "singular coarsest-grid matrix";
    case PD_ERR_STATE: return "call not valid for this context";
  }
  return "unknown status";
}

const char *pd_last_error(const pd_ctx *c) { return c ? c->err.c_str() : ""; }

pd_status pd_allatonce_residual32(pd_ctx *c, float *r32, const double *u, const double *f,
                                  const double *u0, double *h_norms) {
  if (!c || !r32 || !u || !f) return PD_ERR_ARG;
  if (!c->have_B || c->cfg.precision != 1) return PD_ERR_STATE;
  PD_TRY(c, {
    double rn, fn;
    if (c->bidiag) {
      allatonce_norms(c, nullptr, u, f, u0, &rn, &fn, r32, -1.0);
    } else {
      // general B: the FP64 residual, then rounded
      allatonce_norms(c, c->d_r, u, f, u0, &rn, &fn);
      launch_round_to_float(c->stream, (long long)c->n * c->N * c->N, c->d_r, r32);
      ck_launch(c);
      ck(c, cudaStreamSynchronize(c->stream));
    }
    if (h_norms) {
      h_norms[0] = rn;
      h_norms[1] = fn;
    }
    return PD_OK;
  })
}

pd_status pd_shifted_residual32(pd_ctx *c, float *r32, const void *z, const void *b, double *h_norms) {
  if (!c || !r32 || !z || !b) return PD_ERR_ARG;
  if (c->cfg.precision != 1) return PD_ERR_STATE;
  PD_TRY(c, {
    const int N = c->N, n = c->n, gx = shift_residual_blocks(N, n, c->num_sms);
    const double h = hl(c, 0);
    for (int j = 0; j < n; j++) c->h_rsc[j] = 1.0f;
    ck(c, cudaMemcpyAsync(c->d_rsc, c->h_rsc, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    const View out = uview(r32, N);
    if (c->cfg.fx_residual)
      launch_shift_residual_fx(c->stream, gx, N, n, static_cast<const double2 *>(z),
                               static_cast<const double2 *>(b), c->d_lam, c->kappa / (h * h), 1.0f,
                               c->d_rsc, out, nullptr, c->d_srpart);
    else
      launch_shift_residual(c->stream, gx, N, n, static_cast<const double2 *>(z),
                            static_cast<const double2 *>(b), c->d_c1, c->kappa / (h * h), 1.0f, c->d_rsc,
                            out, nullptr, false, c->d_srpart);
    ck_launch(c, c->cfg.fx_residual ? 2 : 1);
    ck(c, cudaMemcpyAsync(c->h_srpart, c->d_srpart, (size_t)n * gx * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    ck(c, cudaStreamSynchronize(c->stream));
    if (h_norms)
      for (int j = 0; j < n; j++) {
        double sum = 0.0;
        for (int x = 0; x < gx; x++) sum += c->h_srpart[(size_t)j * gx + x];
        h_norms[j] = std::sqrt(sum);
      }
    return PD_OK;
  })
}

pd_status shifted_solve_refined(pd_ctx *c, void *z, const void *b, int *h_iters, double *h_relres) {
  if (!c || !z || !b) return PD_ERR_ARG;
  if (c->cfg.precision == 0) return shifted_solve_batched(c, z, b, h_iters, h_relres);
  PD_TRY(c, {
    std::vector<RefRun> runs(1);
    runs[0].c = c;
    runs[0].z = static_cast<double2 *>(z);
    runs[0].b = static_cast<const double2 *>(b);
    refine_runs(runs);
    ck(c, cudaStreamSynchronize(c->stream));
    check_wait_flags(c);
    for (int j = 0; j < c->n; j++) {
      if (h_iters) h_iters[j] = runs[0].it_sum.empty() ? 0 : runs[0].it_sum[j];
      if (h_relres) h_relres[j] = runs[0].relres.empty() ? 0.0 : runs[0].relres[j];
    }
    return runs[0].rc;
  })
}

}  // extern "C"

struct pd_batch {
  std::vector<pd_ctx *> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  cudaStream_t user = nullptr;
  std::string err;
  BatchPlan plan;  // batched launches over all instances (all instances share one stream)
};

namespace {

void free_batch(pd_batch *bt) {
  for (cudaStream_t s : bt->streams)
    if (s) cudaStreamSynchronize(s);
  free_plan(bt->plan);
  for (pd_ctx *c : bt->ctx) free_ctx(c);
  for (cudaEvent_t e : bt->done)
    if (e) cudaEventDestroy(e);
  if (bt->fork) cudaEventDestroy(bt->fork);
  for (cudaStream_t s : bt->streams)
    if (s) cudaStreamDestroy(s);
  delete bt;
}

}  // namespace

extern "C" {

pd_status pd_batch_setup(pd_batch **out, int count, const int *h_N, const int *h_n,
                         const double *const *h_shifts, const pd_config *cfg_in, void *stream) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if (count < 1 || count > 64 || !h_N || !h_n || !h_shifts) return PD_ERR_ARG;
  pd_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else pd_config_default(&cfg);
  if (cfg.omega_mode == 2) return PD_ERR_ARG;
  for (int i = 0; i < count; i++)
    if (!is_pow2m1(h_N[i]) || h_n[i] < 1 || h_n[i] > kMaxShifts || !h_shifts[i]) return PD_ERR_ARG;
  pd_batch *bt = new (std::nothrow) pd_batch();
  if (!bt) return PD_ERR_NOMEM;
  bt->user = (cudaStream_t)stream;
  // FP32 V(1,1) cycles with the warp-stream kernels: every cycle of all instances in
  // batched launches on one stream; otherwise one stream per instance, cycles side by side
  const bool merge = cfg.precision == 1 && cfg.nu1 == 1 && cfg.nu2 == 1 && cfg.cycle_gamma == 1 &&
                     cfg.fused != 0 && cfg.fused_variant != 1;
  if (merge) cfg.fused_variant = 2;
  // one stream per instance, and in batched mode one more for the batched cycles
  const int nstreams = merge ? count + 1 : count;
  bt->streams.assign(nstreams, nullptr);
  bt->done.assign(nstreams, nullptr);
  auto fail = [&](pd_status st) {
    free_batch(bt);
    return st;
  };
  if (cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(PD_ERR_CUDA);
  }
  for (int i = 0; i < nstreams; i++)
    if (cudaStreamCreateWithFlags(&bt->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->done[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(PD_ERR_CUDA);
    }
  for (int i = 0; i < count; i++) {
    pd_ctx *c = nullptr;
    const pd_status st = paradiag_setup(&c, h_N[i], 1.0 / (h_N[i] + 1), h_n[i], h_shifts[i], nullptr,
                                        nullptr, nullptr, nullptr, nullptr, &cfg, bt->streams[i]);
    if (st != PD_OK) return fail(st);
    bt->ctx.push_back(c);
  }
  if (merge) {
    bt->plan.ctx = bt->ctx;
    bt->plan.stream = bt->streams[count];
    try {
      build_plan(bt->plan);
    } catch (const CudaFail &) {
      bt->err = bt->ctx[0]->err;
      return fail(PD_ERR_CUDA);
    }
  }
  *out = bt;
  return PD_OK;
}

pd_status pd_batch_solve(pd_batch *bt, void *const *d_z, const void *const *d_b, int *h_iters,
                         double *h_relres) {
  if (!bt || !d_z || !d_b) return PD_ERR_ARG;
  const size_t k = bt->ctx.size();
  for (size_t i = 0; i < k; i++)
    if (!d_z[i] || !d_b[i]) return PD_ERR_ARG;
  pd_ctx *c0 = bt->ctx[0];
  pd_ctx *c = c0;  // context whose error text a failure reports
  try {
    ck(c0, cudaEventRecord(bt->fork, bt->user));
    for (size_t i = 0; i < bt->streams.size(); i++) ck(c0, cudaStreamWaitEvent(bt->streams[i], bt->fork, 0));
    std::vector<pd_status> rc(k, PD_OK);
    std::vector<std::vector<int>> its(k);
    std::vector<std::vector<double>> rel(k);
    if (c0->cfg.precision == 0) {
      for (size_t i = 0; i < k; i++) {
        c = bt->ctx[i];
        LevelBufs &B = c->p64.lv[0];
        launch_copy_scale<double>(c->stream, c->N, c->n, view(B.b, c->N, B.P), uview(d_b[i], c->N),
                                  rs(c, 0));
        ck_launch(c);
      }
      c = c0;
      lockstep_solve<double>(bt->ctx, false, rc);
      for (size_t i = 0; i < k; i++) {
        c = bt->ctx[i];
        LevelBufs &B = c->p64.lv[0];
        launch_gather_final<double>(c->stream, c->N, c->n, uview(d_z[i], c->N),
                                    view(B.z[0], c->N, B.P), view(B.z[1], c->N, B.P),
                                    c->st.final_buf);
        ck_launch(c);
        its[i].assign(c->h_iters, c->h_iters + c->n);
        rel[i].assign(c->h_relres, c->h_relres + c->n);
      }
    } else {
      std::vector<RefRun> runs(k);
      for (size_t i = 0; i < k; i++) {
        runs[i].c = bt->ctx[i];
        runs[i].z = static_cast<double2 *>(d_z[i]);
        runs[i].b = static_cast<const double2 *>(d_b[i]);
      }
      refine_runs(runs, bt->plan.ok ? &bt->plan : nullptr);
      for (size_t i = 0; i < k; i++) {
        rc[i] = runs[i].rc;
        its[i] = runs[i].it_sum;
        rel[i] = runs[i].relres;
      }
    }
    for (size_t i = 0; i < bt->streams.size(); i++) {
      ck(c0, cudaEventRecord(bt->done[i], bt->streams[i]));
      ck(c0, cudaStreamWaitEvent(bt->user, bt->done[i], 0));
    }
    for (size_t i = 0; i < k; i++) {
      c = bt->ctx[i];
      check_wait_flags(c);
    }
    size_t o = 0;
    pd_status out = PD_OK;
    for (size_t i = 0; i < k; i++) {
      const int n = bt->ctx[i]->n;
      for (int j = 0; j < n; j++, o++) {
        if (h_iters) h_iters[o] = its[i].empty() ? 0 : its[i][j];
        if (h_relres) h_relres[o] = rel[i].empty() ? 0.0 : rel[i][j];
      }
      if (out == PD_OK && rc[i] != PD_OK) {
        out = rc[i];
        bt->err = "instance " + std::to_string(i) + ": " + pd_status_str(rc[i]);
      }
    }
    return out;
  } catch (const CudaFail &) {
    bt->err = c->err;
    return PD_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    bt->err = "out of memory";
    return PD_ERR_NOMEM;
  } catch (pd_status st) {
    bt->err = pd_status_str(st);
    return st;
  }
}

pd_status pd_batch_destroy(pd_batch *bt) {
  if (!bt) return PD_ERR_ARG;
  free_batch(bt);
  return PD_OK;
}

const char *pd_batch_last_error(const pd_batch *bt) { return bt ? bt->err.c_str() : ""; }

pd_status pd_batch_info(const pd_batch *bt, int *h_batched, int *h_launches_per_cycle, long long *h_launches) {
  if (!bt) return PD_ERR_ARG;
  const BatchPlan &bp = bt->plan;
  if (h_batched) *h_batched = bp.ok ? 1 : 0;
  if (h_launches_per_cycle) *h_launches_per_cycle = bp.ok ? 2 * bp.gmax + 2 : -1;
  if (h_launches) *h_launches = bp.launches;
  return PD_OK;
}

long long pd_batch_launch_count(const pd_batch *bt) {
  if (!bt) return 0;
  long long n = bt->plan.launches;
  for (const pd_ctx *c : bt->ctx) n += c->launches;
  return n;
}

}  // extern "C"
