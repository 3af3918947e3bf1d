// liblcmg: host runtime and C ABI (see include/lcmg.h).
//
// The context owns the forward operator (CSR A and its transpose, or a
// PSF), the edge weights, the lambda-independent Galerkin hierarchy and a
// workspace sized for the widest batch seen.  A solve advances all
// (lambda, right-hand side) columns of a batch together: every PCG
// iteration is a fixed sequence of kernel launches whose per-column
// scalars (alpha, beta, convergence) stay on the device; the host polls a
// few counters every `check_every` iterations, and then runs the
// true-residual check (and, on the mixed path, the reliable update) in
// FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "launch.h"
#include "vfused.cuh"
#include "paper_mg.cuh"
#include "rs_amg.h"
#include "lcmg.h"

namespace lcmg {

static thread_local std::string g_err;

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  // grow-only allocation of at least cnt elements
  T* need(size_t cnt) {
    if (cnt == 0) cnt = 1;
    if (p && n >= cnt) return p;
    release();
    void* q = nullptr;
    if (cudaMalloc(&q, cnt * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      throw MemError("device allocation of " + std::to_string(cnt * sizeof(T)) + " bytes failed");
    }
    p = static_cast<T*>(q);
    n = cnt;
    return p;
  }
};

struct Level {
  int nv = 0, nh = 0;
  int64_t n = 0;
  DevBuf<double> gl, ga;   // 25 x n (levels >= 1)
  DevBuf<double> cf64;     // per-point coefficient rows (smoother layout)
  DevBuf<float> cf32;
  // FP16 smoother data (levels >= 1): per-lambda rows of K's off-diagonals,
  // the row sums of G_A, and the largest off-diagonal |G_L|, |G_A| (scales)
  DevBuf<__half> hrows;
  DevBuf<float> hs;
  double glmax = 0.0, gamax = 0.0;
  double hscale = 1.0;     // scale of the rows of the current lambda
};

struct LevelWork {
  DevBuf<char> rhs, z, t, res, dinv;  // T-typed, n_k x B
};

// One level of the paper's one-sided hierarchy (params.precond = 1):
// A_k (rows of A, n_k columns) and its transpose, FP64, and diag(A_k^T A_k).
// Level 0 uses the forward operator itself.
struct PmLevel {
  int64_t nnz = 0;
  DevBuf<int64_t> rp, rpT;
  DevBuf<int32_t> ci, ciT;
  DevBuf<double> v, vT, dA;
};

// A level of the classical AMG hierarchy on the device (params.coarsening =
// 1): P_k (n_k x n_{k+1}) and P_k^T as CSR, and G_L^k = M_k^T M_k as CSR with
// its diagonal (levels k >= 1).
struct AmLevel {
  int64_t n = 0;
  DevBuf<int64_t> prp, ptrp, grp;
  DevBuf<int32_t> pci, ptci, gci;
  DevBuf<double> pv, ptv, gv, gdiag;
};

// One-column workspace of a level of the paper's cycle.
struct PmWork {
  DevBuf<double> b, x, r, z, p, q, t, y, dinv, pa, pb, ppq;
};

constexpr int kMaxBlocks = 2048;
// widest batch for which params.vfuse = 1 picks the two-kernels-per-level
// V-cycle (its blocks read one column each: wider batches read strided)
constexpr int kVfuseAutoB = 4;

// Choices of the autotuner for one batch width (params.autotune): the
// one-column SpMV configuration of each operator pass (SpmmArgs::variant)
// and the V-cycle form (1 = two kernels per level, 0 = one per step).
struct Tuned {
  int var_a = 0, var_at = 0, vfuse = -1;
};

}  // namespace lcmg

using namespace lcmg;

struct lcmg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  lcmg_params prm{};
  int sms = 0;
  int maxblk = 0;
  // grid
  int nv = 0, nh = 0;
  int64_t n = 0, ne = 0;
  // forward operator
  int fwd = 0;  // 0 none, 1 CSR, 2 PSF
  int64_t m = 0, nnz = 0;
  int vdtype = 0;  // 0 FP32 values, 1 FP64 values
  DevBuf<int64_t> rp, rpT;
  DevBuf<int32_t> ci, ciT;
  DevBuf<float> v32, vT32;
  DevBuf<double> v64, vT64;
  // 16-bit column offsets from a per-row base (A and A^T), when every row's
  // column span fits: read by the one-column SpMV
  DevBuf<uint16_t> c16, c16T;
  DevBuf<int32_t> rbase, rbaseT;
  bool c16_ok = false;
  DevBuf<double> ones;   // n ones (unweighted gradient norm)
  bool ones_ok = false;
  std::map<int, lcmg::Tuned> tuned;  // autotuner choices per (batch width, precision)
  // the paper's own preconditioner (params.precond = 1)
  std::vector<lcmg::PmLevel> pm;
  std::vector<lcmg::PmWork> pmw;
  DevBuf<double> pm_AtAc;            // dense A_c^T A_c of the coarsest level
  int pm_levels = 0;                 // levels the one-sided hierarchy was built for (0: none)
  std::vector<lcmg::AmLevel> am;     // classical AMG levels (params.coarsening = 1)
  bool am_ok = false;                // am and pm hold the AMG hierarchy of the current D
  DevBuf<double> pm_GLc;             // dense G_L^c of the coarsest AMG level
  DevBuf<double> pm_V, pm_Z, pm_w, pm_r, pm_h, pm_part, pm_y;
  DevBuf<double> pm_cin, pm_cout;    // input and output of the captured cycle
  int rv = 0, rh = 0;
  DevBuf<double> psf64;
  DevBuf<float> psf32;
  // separable PSF fv fh^T (sep): the banded passes of A^T A along i and j
  // (with their boundary correction rows in FP64 and FP32), of A and of A^T
  bool sep = false;
  lcmg::SepPass sp_vt, sp_ht, sp_va, sp_ha, sp_vat, sp_hat;
  DevBuf<double> sep_dv64, sep_dh64;
  DevBuf<float> sep_dv32, sep_dh32;
  DevBuf<double> sep_tmp;  // intermediate of A^T b and of rho = ||A x - b||
  DevBuf<double> diag;
  DevBuf<float> diag32;
  // weights
  DevBuf<double> d, ws, we;
  DevBuf<float> ws32, we32;
  // FP16 copies of the finest level's smoother data (w_s, w_e scaled by
  // hw_scale, diag(A^T A) by hg_scale); h16_on: the current batch uses them
  DevBuf<__half> h_ws, h_we, h_ga;
  double hw_scale = 1.0, hg_scale = 1.0;
  DevBuf<unsigned long long> hmax;
  bool h16_on = false;
  // hierarchy
  std::vector<Level> lev;
  bool hier_ok = false;
  // workspace
  int Bcap = 0;
  DevBuf<double> x64, c64, r64, y64, bvec, cvec;
  DevBuf<float> xlo;
  DevBuf<char> r, z, p, q, y;
  std::vector<LevelWork> lw;
  DevBuf<double> lam2;
  DevBuf<char> lam2T;
  DevBuf<double> kinv, Mw, Ww;
  DevBuf<double> part_pq, part_rr, part_rz, part_x;
  DevBuf<double> s_rz, s_rz2, s_alpha, s_beta, s_rr, s_rmax, s_tol2cc, s_cc, s_rrtrue, s_out;
  DevBuf<int> s_active, s_iters, s_status, s_pending, s_counters, s_info, s_flag;
  DevBuf<double*> colptr;
  DevBuf<int> colmap;
  int* h_counters = nullptr;  // pinned
  // weight-update scratch
  DevBuf<double> absv, bmax;
  // events of the operator-pass timing (params.timing)
  std::vector<cudaEvent_t> tev;
  int tev_used = 0;
  // staging for host-pointer calls and the outer loop (grow-only: no
  // allocation in steady state)
  DevBuf<double> stage_b, stage_x, stage_x0, run_xres, run_xstar, run_xwin;
  lcmg_stats stats{};
};

namespace lcmg {

static void set_err(const std::string& s) { g_err = s; }

// Copies and fills go on the context's stream and are waited for there:
// the legacy default stream would synchronise implicitly with every
// blocking stream of the process, including a stream that another thread
// is capturing into a CUDA graph (several contexts serve in parallel).
static void copy_sync(cudaStream_t s, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  LCMG_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, s));
  LCMG_CUDA(cudaStreamSynchronize(s));
}
static void fill_sync(cudaStream_t s, void* dst, int v, size_t bytes) {
  LCMG_CUDA(cudaMemsetAsync(dst, v, bytes, s));
  LCMG_CUDA(cudaStreamSynchronize(s));
}

// SpMM arguments for A (trans false) or A^T over ld interleaved columns
static SpmmArgs csr_args(const lcmg_ctx& c, bool trans, int ld) {
  SpmmArgs a{};
  a.rows = trans ? c.n : c.m;
  a.rp = trans ? c.rpT.p : c.rp.p;
  a.ci = trans ? c.ciT.p : c.ci.p;
  a.B = ld; a.c0 = 0; a.nb = ld; a.nl = 1; a.nrhs = 1;
  if (c.c16_ok && c.prm.compact_cols) {
    a.c16 = trans ? c.c16T.p : c.c16.p;
    a.rbase = trans ? c.rbaseT.p : c.rbase.p;
  }
  return a;
}

// for entry points defined in other translation units
void set_error_message(const std::string& s) { g_err = s; }

static void check_params(const lcmg_params& p) {
  if (p.levels < 0 || p.coarse_max < 1 || p.nu < 1 || p.nu > 16) throw ArgError("invalid levels/coarse_max/nu");
  if (p.smoother != LCMG_SMOOTH_L1_JACOBI && p.smoother != LCMG_SMOOTH_JACOBI) throw ArgError("invalid smoother");
  if (!(p.omega > 0.0 && p.omega < 2.0)) throw ArgError("omega must lie in (0, 2)");
  if (!(p.q > 0.0) || !(p.d_min > 0.0 && p.d_min <= 1.0)) throw ArgError("q must be > 0 and d_min in (0, 1]");
  if (!(p.tol > 0.0 && p.tol < 1.0) || p.maxit < 1) throw ArgError("tol must lie in (0, 1) and maxit >= 1");
  if (p.precision != LCMG_PREC_FP64 && p.precision != LCMG_PREC_MIXED) throw ArgError("invalid precision");
  if (p.mode != LCMG_MODE_BATCHED && p.mode != LCMG_MODE_SEQUENTIAL) throw ArgError("invalid mode");
  if (p.check_every < 1) throw ArgError("check_every must be >= 1");
  if (p.vfuse < 0 || p.vfuse > 2) throw ArgError("vfuse must be 0, 1 or 2");
  if (p.keep_direction != 0 && p.keep_direction != 1) throw ArgError("keep_direction must be 0 or 1");
  if (p.autotune != 0 && p.autotune != 1) throw ArgError("autotune must be 0 or 1");
  if (p.spmv_variant < 0 || p.spmv_variant > 6) throw ArgError("spmv_variant must be 0..6");
  if (p.spmv_variant_at < 0 || p.spmv_variant_at > 6) throw ArgError("spmv_variant_at must be 0..6");
  if (p.stop_rule != 0 && p.stop_rule != 1) throw ArgError("stop_rule must be 0 or 1");
  if (p.precond != 0 && p.precond != 1) throw ArgError("precond must be 0 or 1");
  if (p.gmres_restart < 1 || p.gmres_restart > 2000) throw ArgError("gmres_restart must be 1..2000");
  if (p.coarsening < 0 || p.coarsening > 2) throw ArgError("coarsening must be 0, 1 or 2");
  if (p.compact_cols != 0 && p.compact_cols != 1) throw ArgError("compact_cols must be 0 or 1");
  if (p.alpha_fuse != 0 && p.alpha_fuse != 1) throw ArgError("alpha_fuse must be 0 or 1");
  if (p.beta_fuse != 0 && p.beta_fuse != 1) throw ArgError("beta_fuse must be 0 or 1");
  if (p.amg_coarse_max < 2 || p.amg_coarse_max > 2048) throw ArgError("amg_coarse_max must be 2..2048");
  if (p.max_blocks < 0) throw ArgError("max_blocks must be >= 0");
  if (p.smoother_fp16 != 0 && p.smoother_fp16 != 1) throw ArgError("smoother_fp16 must be 0 or 1");
}

static int sum_blocks(int nb) { return std::max(1, std::min(nb, kMaxBlocks)); }

// ---------------------------------------------------------------------------
// Hierarchy
// ---------------------------------------------------------------------------
static int level_count(const lcmg_ctx& c) {
  // with classical AMG `levels` bounds the AMG hierarchy; the geometric one
  // (used by the default preconditioner) then takes its default depth
  if (c.prm.levels > 0 && c.prm.coarsening == 0) return c.prm.levels;
  int lv = 1, a = c.nv, b = c.nh;
  while ((a > c.prm.coarse_max || b > c.prm.coarse_max) && a % 2 == 0 && b % 2 == 0) {
    a /= 2; b /= 2; ++lv;
  }
  return lv;
}

static void refresh_fine(lcmg_ctx& c) {
  const int g = (int)std::min<int64_t>((c.n + kBlock - 1) / kBlock, c.maxblk);
  klaunch(k_edge_to_pixel, dim3(g), dim3(kBlock), 0, c.stream, c.nv, c.nh, c.d.p, c.ws.need(c.n), c.we.need(c.n));
  LCMG_LAUNCHED();
  klaunch(k_convert<double, float>, dim3(g), dim3(kBlock), 0, c.stream, c.n, c.ws.p, c.ws32.need(c.n));
  LCMG_LAUNCHED();
  klaunch(k_convert<double, float>, dim3(g), dim3(kBlock), 0, c.stream, c.n, c.we.p, c.we32.need(c.n));
  LCMG_LAUNCHED();
  c.hier_ok = false;
  c.am_ok = false;  // classical AMG coarsens L^T D^2 L: rebuilt for every D
}

// The lambda-independent part of the FP16 smoother data: the finest
// level's w_s, w_e, diag(A^T A) in FP16 with their scales, and per coarse
// level the FP32 row sums of G_A and the largest off-diagonal |G_L|, |G_A|
// (the scale of a lambda's rows: lam^2 glmax + gamax bounds |K|'s entries)
static void build_half(lcmg_ctx& c) {
  const int L = (int)c.lev.size();
  unsigned long long* mx = c.hmax.need(2 * L + 2);
  LCMG_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * (2 * L + 2), c.stream));
  const int g0 = (int)std::min<int64_t>((c.n + kBlock - 1) / kBlock, c.maxblk);
  klaunch(k_maxabs, dim3(g0), dim3(kBlock), 0, c.stream, c.n, (const double*)c.ws.p, 0, mx);
  LCMG_LAUNCHED();
  klaunch(k_maxabs, dim3(g0), dim3(kBlock), 0, c.stream, c.n, (const double*)c.we.p, 0, mx);
  LCMG_LAUNCHED();
  klaunch(k_maxabs, dim3(g0), dim3(kBlock), 0, c.stream, c.n, (const double*)c.diag.p, 0, mx + 1);
  LCMG_LAUNCHED();
  for (int k = 1; k < L; ++k) {
    Level& g = c.lev[k];
    const int gk = (int)std::min<int64_t>((g.n + kBlock - 1) / kBlock, c.maxblk);
    klaunch(k_maxabs, dim3(gk), dim3(kBlock), 0, c.stream, g.n, (const double*)g.gl.p, 1, mx + 2 * k);
    LCMG_LAUNCHED();
    klaunch(k_maxabs, dim3(gk), dim3(kBlock), 0, c.stream, g.n, (const double*)g.ga.p, 1, mx + 2 * k + 1);
    LCMG_LAUNCHED();
    klaunch(k_rowsum25, dim3(gk), dim3(kBlock), 0, c.stream, g.n, (const double*)g.ga.p, g.hs.need(g.n));
    LCMG_LAUNCHED();
    g.hrows.need((size_t)kCompactOff * g.n);
  }
  std::vector<unsigned long long> hm(2 * L + 2);
  copy_sync(c.stream, hm.data(), mx, sizeof(unsigned long long) * hm.size(), cudaMemcpyDeviceToHost);
  auto dbl = [](unsigned long long b) { double v; std::memcpy(&v, &b, sizeof v); return v; };
  c.hw_scale = half_scale(dbl(hm[0]));
  c.hg_scale = half_scale(dbl(hm[1]));
  for (int k = 1; k < L; ++k) {
    c.lev[k].glmax = dbl(hm[2 * k]);
    c.lev[k].gamax = dbl(hm[2 * k + 1]);
  }
  klaunch(k_half_scaled, dim3(g0), dim3(kBlock), 0, c.stream, c.n, (const double*)c.ws.p, c.hw_scale, c.h_ws.need(c.n));
  LCMG_LAUNCHED();
  klaunch(k_half_scaled, dim3(g0), dim3(kBlock), 0, c.stream, c.n, (const double*)c.we.p, c.hw_scale, c.h_we.need(c.n));
  LCMG_LAUNCHED();
  klaunch(k_half_scaled, dim3(g0), dim3(kBlock), 0, c.stream, c.n, (const double*)c.diag.p, c.hg_scale,
          c.h_ga.need(c.n));
  LCMG_LAUNCHED();
}

static void build_hierarchy(lcmg_ctx& c) {
  if (c.fwd == 0) throw ArgError("forward operator not set");
  const int L = level_count(c);
  int a = c.nv, b = c.nh;
  for (int k = 1; k < L; ++k) {
    if (a % 2 || b % 2) throw ArgError("grid sides must be divisible by 2^(levels-1)");
    a /= 2; b /= 2;
  }
  const int64_t nc = (int64_t)a * b;
  if (nc > 4096) throw ArgError("coarsest level has " + std::to_string(nc) + " unknowns (dense limit 4096): use more levels");
  c.lev.resize(L);
  c.lev[0].nv = c.nv; c.lev[0].nh = c.nh; c.lev[0].n = c.n;
  for (int k = 1; k < L; ++k) {
    Level& f = c.lev[k - 1];
    Level& g = c.lev[k];
    g.nv = f.nv / 2; g.nh = f.nh / 2; g.n = (int64_t)g.nv * g.nh;
    double* gl = g.gl.need(kStencil * g.n);
    double* ga = g.ga.need(kStencil * g.n);
    RapIn in{};
    in.nvf = f.nv; in.nhf = f.nh; in.nf = f.n;
    if (k == 1) {
      in.ws = c.ws.p; in.we = c.we.p; in.ga = c.diag.p;
      in.part = 0; launch_galerkin(in, g.nv, g.nh, gl, c.maxblk, c.stream);
      in.part = 1; launch_galerkin(in, g.nv, g.nh, ga, c.maxblk, c.stream);
    } else {
      in.part = 2;
      in.g25 = f.gl.p; launch_galerkin(in, g.nv, g.nh, gl, c.maxblk, c.stream);
      in.g25 = f.ga.p; launch_galerkin(in, g.nv, g.nh, ga, c.maxblk, c.stream);
    }
    // smoother copies: per-point rows of both parts (FP64 and FP32)
    const int gg = (int)std::min<int64_t>((kCoefStride * g.n + kBlock - 1) / kBlock, c.maxblk);
    klaunch(k_coef_pack<double>, dim3(gg), dim3(kBlock), 0, c.stream, g.n, gl, ga, g.cf64.need(kCoefStride * g.n));
    LCMG_LAUNCHED();
    klaunch(k_coef_pack<float>, dim3(gg), dim3(kBlock), 0, c.stream, g.n, gl, ga, g.cf32.need(kCoefStride * g.n));
    LCMG_LAUNCHED();
  }
  build_half(c);
  c.hier_ok = true;
}

static void ensure_hierarchy(lcmg_ctx& c) {
  if (!c.hier_ok) build_hierarchy(c);
}

template <class T>
static LevelView<T> view(const lcmg_ctx& c, int k);
template <>
LevelView<double> view<double>(const lcmg_ctx& c, int k) {
  LevelView<double> v;
  const Level& l = c.lev[k];
  v.nv = l.nv; v.nh = l.nh; v.n = l.n;
  if (k == 0) { v.fine = true; v.ws = c.ws.p; v.we = c.we.p; v.ga = c.diag.p; }
  else { v.fine = false; v.cf = l.cf64.p; }
  return v;
}
template <>
LevelView<float> view<float>(const lcmg_ctx& c, int k) {
  LevelView<float> v;
  const Level& l = c.lev[k];
  v.nv = l.nv; v.nh = l.nh; v.n = l.n;
  if (k == 0) { v.fine = true; v.ws = c.ws32.p; v.we = c.we32.p; v.ga = c.diag32.p; }
  else { v.fine = false; v.cf = l.cf32.p; }
  if (c.h16_on) {
    v.h16 = true;
    v.fh = FineOpH{l.nv, l.nh, c.h_ws.p, c.h_we.p, c.h_ga.p, (float)(1.0 / c.hw_scale), (float)(1.0 / c.hg_scale)};
    v.ch = CoarseOpH{l.nv, l.nh, l.n, reinterpret_cast<const uint4*>(l.hrows.p), l.hs.p, (float)(1.0 / l.hscale)};
  }
  return v;
}

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
static void ensure_work(lcmg_ctx& c, int B) {
  const size_t nB = (size_t)c.n * B, mB = (size_t)c.m * B;
  c.x64.need(nB); c.c64.need(nB); c.r64.need(nB); c.y64.need(std::max(mB, nB));
  c.xlo.need(nB);
  const size_t tb = sizeof(double);  // room for either precision
  c.r.need(nB * tb); c.z.need(nB * tb); c.p.need(nB * tb); c.q.need(nB * tb);
  c.y.need(std::max(mB, nB) * tb);
  const int L = (int)c.lev.size();
  c.lw.resize(L);
  for (int k = 0; k < L; ++k) {
    const size_t nk = (size_t)c.lev[k].n * B * tb;
    c.lw[k].t.need(nk); c.lw[k].res.need(nk); c.lw[k].dinv.need(nk);
    if (k > 0) { c.lw[k].rhs.need(nk); c.lw[k].z.need(nk); }
  }
  const size_t nc = (size_t)c.lev[L - 1].n;
  c.kinv.need(nc * nc * B); c.Mw.need(nc * nc * B); c.Ww.need(nc * nc * B);
  c.lam2.need(B); c.lam2T.need(B * tb);
  const size_t pb = (size_t)kMaxBlocks * B;
  c.part_pq.need(pb); c.part_rr.need(pb); c.part_rz.need(pb); c.part_x.need(pb);
  for (auto* b : {&c.s_rz, &c.s_rz2, &c.s_alpha, &c.s_beta, &c.s_rr, &c.s_rmax, &c.s_tol2cc, &c.s_cc, &c.s_rrtrue, &c.s_out})
    b->need(B);
  for (auto* b : {&c.s_active, &c.s_iters, &c.s_status, &c.s_pending, &c.s_info, &c.s_flag}) b->need(B);
  c.s_counters.need(4);
  if (!c.h_counters) LCMG_CUDA(cudaMallocHost(&c.h_counters, 4 * sizeof(int)));
  c.Bcap = std::max(c.Bcap, B);
}

static ColState colstate(lcmg_ctx& c) {
  ColState s;
  s.rz = c.s_rz.p; s.rz2 = c.s_rz2.p; s.alpha = c.s_alpha.p; s.beta = c.s_beta.p; s.rr = c.s_rr.p; s.rmax = c.s_rmax.p;
  s.tol2cc = c.s_tol2cc.p; s.active = c.s_active.p; s.iters = c.s_iters.p; s.status = c.s_status.p;
  s.pending = c.s_pending.p; s.counters = c.s_counters.p;
  s.keep = c.prm.keep_direction ? 1 : 0;
  return s;
}

// ---------------------------------------------------------------------------
// Batched solver for one precision T (double: FP64 path; float: mixed)
// ---------------------------------------------------------------------------
template <class T>
static void op_bytes(const lcmg_ctx& c, int B, int64_t* first, int64_t* second);

template <class T>
struct Batch {
  lcmg_ctx& c;
  int B;
  cudaStream_t s;
  int nlev;

  // autotuned or forced choices (0 / -1: the defaults)
  int var_a = 0, var_at = 0, vf_force = -1;
  int tune_key() const { return 2 * B + (std::is_same<T, float>::value ? 1 : 0); }

  Batch(lcmg_ctx& c_, int B_) : c(c_), B(B_), s(c_.stream), nlev((int)c_.lev.size()) {
    c.h16_on = false;
    var_a = var_at = c.prm.spmv_variant;
    if (c.prm.spmv_variant_at) var_at = c.prm.spmv_variant_at;
    auto it = c.tuned.find(tune_key());
    if (c.prm.autotune && it != c.tuned.end()) {
      var_a = it->second.var_a;
      var_at = it->second.var_at;
      vf_force = it->second.vfuse;
    }
  }

  ~Batch() { c.h16_on = false; }
  Batch(const Batch&) = delete;
  Batch& operator=(const Batch&) = delete;

  T* tp(DevBuf<char>& b) { return reinterpret_cast<T*>(b.p); }

  // the finest level of the two-kernels-per-level V(1,1) cycle with FP32
  // vectors runs k_vfine_down / k_vfine_up
  bool fine_v11() const { return std::is_same<T, float>::value && c.prm.nu == 1 && vf_on(); }

  // the two-kernels-per-level V-cycle runs for this batch
  bool vf_on() const {
    const int nu = c.prm.nu;
    const bool vf = vf_force >= 0 ? vf_force == 1 : (c.prm.vfuse == 2 || (c.prm.vfuse == 1 && B <= kVfuseAutoB));
    return nlev >= 2 && vf && (nu == 1 || nu == 2);
  }
  const T* lam2T() { return reinterpret_cast<const T*>(c.lam2T.p); }
  FineOp<T> fop() { return view<T>(c, 0).fine_op(); }
  FineOp<double> fop64() { return view<double>(c, 0).fine_op(); }

  SpmmArgs args(bool trans, int ld) { return csr_args(c, trans, ld); }
  PsfArgs psf() {
    PsfArgs a{};
    a.nv = c.nv; a.nh = c.nh; a.rv = c.rv; a.rh = c.rh; a.psf = c.psf64.p;
    return a;
  }
  const T* psfT();
  // banded passes of the separable A^T A in precision T (correction rows of
  // the matching precision)
  Band<T> band_vt() {
    return make_band<T>(c.sp_vt, std::is_same<T, double>::value ? reinterpret_cast<const T*>(c.sep_dv64.p)
                                                                : reinterpret_cast<const T*>(c.sep_dv32.p));
  }
  Band<T> band_ht() {
    return make_band<T>(c.sp_ht, std::is_same<T, double>::value ? reinterpret_cast<const T*>(c.sep_dh64.p)
                                                                : reinterpret_cast<const T*>(c.sep_dh32.p));
  }

  // q = K p (T precision) with partials of p.q; returns the partial count
  int apply_K(const T* P, T* Q, double* part);

  // ---- live timing of the operator passes (params.timing) ------------
  // Only the first iteration of each block of check_every iterations is
  // bracketed by events (a sample: the event-record nodes themselves cost
  // time inside the graph).
  bool timing_now = false;
  void mark() {
    if (!c.prm.timing || !timing_now) return;
    if (c.tev_used >= (int)c.tev.size()) {
      cudaEvent_t e;
      LCMG_CUDA(cudaEventCreate(&e));
      c.tev.push_back(e);
    }
    // External: inside a stream capture this becomes an event-record node
    // of the graph (a plain record would only express a dependency)
    LCMG_CUDA(cudaEventRecordWithFlags(c.tev[c.tev_used++], s, cudaEventRecordExternal));
  }
  // after the stream has been synchronised: add the recorded pass and
  // V-cycle times (five events per timed iteration: the two operator
  // passes, then the V-cycle)
  void collect_timing() {
    if (!c.prm.timing) return;
    int64_t b0 = 0, b1 = 0;
    op_bytes<T>(c, B, &b0, &b1);
    const int64_t vb = vcycle_bytes();
    for (int i = 0; i + 4 < c.tev_used; i += 5) {
      float a = 0.f, b = 0.f, v = 0.f;
      if (cudaEventElapsedTime(&a, c.tev[i], c.tev[i + 1]) != cudaSuccess ||
          cudaEventElapsedTime(&b, c.tev[i + 1], c.tev[i + 2]) != cudaSuccess ||
          cudaEventElapsedTime(&v, c.tev[i + 3], c.tev[i + 4]) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      c.stats.op_ms_a += a;
      c.stats.op_ms_at += b;
      c.stats.op_launches += 2;
      c.stats.op_bytes += b0 + b1;
      c.stats.vcycle_ms += v;
      c.stats.vcycle_count += 1;
      c.stats.vcycle_bytes += vb;
    }
  }
  // Algorithmic DRAM bytes of one V-cycle of this batch in the two-kernels-
  // per-level form: per level k (n_k points, s-byte vectors) the down kernel
  // reads r and dinv and writes the pre-smoothed z and the coarse r (n_k / 4);
  // the up kernel reads the coarse e, the pre-smoothed z, r and dinv and
  // writes z: 7.5 s n_k per column; the smoother data (as stored) is read by
  // both kernels; the coarsest level reads its inverse (n_c^2 doubles per
  // column) and its r and writes its e.
  int64_t vcycle_bytes() const {
    const int64_t sT = sizeof(T);
    int64_t bytes = 0;
    for (int k = 0; k + 1 < nlev; ++k) {
      const int64_t nk = c.lev[k].n;
      int64_t coef = k == 0 ? 3 * sT : (int64_t)kCoefStride * sT;
      if (c.h16_on) coef = k == 0 ? 3 * 2 : kCompactOff * 2 + 4;  // FP16 rows (+ FP32 row sum)
      if (k == 0 && fine_v11()) {
        // r twice, r_c and e_c (a quarter each), z once; no pre-smoothed z, no D^{-1}
        bytes += (nk * 7 / 2) * sT * B + 2 * coef * nk;
        continue;
      }
      bytes += (nk * 15 / 2) * sT * B + 2 * coef * nk;
    }
    const int64_t nc = c.lev[nlev - 1].n;
    bytes += (nc * nc * 8 + 2 * nc * sT) * B;
    return bytes;
  }
  // r64 = c64 - K x64 in FP64 with partials of r64.r64
  int true_residual(double* part);

  // ---- V-cycle (Algorithm 1, gamma = 1, zero initial guess) ----------
  // m Jacobi sweeps z <- z + D^{-1}(rhs - K z), ending in z; with part the
  // r.z partials of the result
  void sweeps(int k, int m, const T* rhs, T* z, T* t, double* part, int* nb_out) {
    if (m <= 0) return;
    LevelView<T> L = view<T>(c, k);
    const T* dinv = tp(c.lw[k].dinv);
    T* a = z;
    T* b = t;
    for (int i = 0; i < m; ++i) {
      const bool last = (i == m - 1);
      const bool with_dot = last && (m % 2 == 0);
      int nb = launch_smooth<T>(L, B, lam2T(), dinv, rhs, a, b, nullptr, with_dot ? part : nullptr,
                                c.maxblk, s);
      if (last && (m % 2 == 0) && nb_out) *nb_out = nb;
      std::swap(a, b);
    }
    if (m % 2 == 1) {  // result is in t: copy back
      launch_copy_cols<T>(L.n, B, nullptr, t, z, c.maxblk, s);
      if (part) {
        const int g = grid_for(L.n, B, c.maxblk);
        klaunch(k_col_dot<T>, dim3(g), dim3(kBlock), 0, s, L.n, B, rhs, z, part);
        LCMG_LAUNCHED();
        if (nb_out) *nb_out = g;
      }
    }
  }

  int vcycle(const T* r0, T* z0, double* part) {
    const int nu = c.prm.nu;
    int nb = 0;
    if (nlev == 1) {
      launch_coarse_solve<T>((int)c.lev[0].n, B, c.kinv.p, r0, z0, s);
      const int g = grid_for(c.n, B, c.maxblk);
      klaunch(k_col_dot<T>, dim3(g), dim3(kBlock), 0, s, c.n, B, r0, z0, part);
      LCMG_LAUNCHED();
      return g;
    }
    std::vector<const T*> rhs(nlev);
    std::vector<T*> zz(nlev);
    rhs[0] = r0; zz[0] = z0;
    for (int k = 1; k < nlev; ++k) { rhs[k] = tp(c.lw[k].rhs); zz[k] = tp(c.lw[k].z); }
    if (vf_on()) {
      // two kernels per level: pre-smoothed z of level k goes to t[k]; the
      // finest level of a V(1,1) cycle in FP32 runs the kernels that form it
      // on the fly (vfine.cuh)
      const bool fine1 = fine_v11();
      // FP16 coarse levels of at most kTailPoints points and the coarsest
      // solve: one single-block kernel (vtail.cuh)
      // (only while the coarsest level is small: its dense FP64 solve then runs
      // on one SM, which at 256 points costs more than the launches saved)
      int t0 = nlev - 1;
      if (std::is_same<T, float>::value && c.h16_on && nu == 1 && c.lev[nlev - 1].n <= kTailCoarsest)
        while (t0 - 1 >= 1 && c.lev[t0 - 1].n <= kTailPoints) --t0;
      if (!vtail_fits(nlev - t0)) t0 = nlev - 1;
      for (int k = 0; k < t0; ++k) {
        if (k == 0 && fine1)
          launch_vfine_down(view<float>(c, 0), B, reinterpret_cast<const float*>(lam2T()), c.prm.smoother,
                            c.prm.omega, reinterpret_cast<const float*>(rhs[0]),
                            reinterpret_cast<float*>(tp(c.lw[1].rhs)), s);
        else
          launch_vdown<T>(view<T>(c, k), B, lam2T(), tp(c.lw[k].dinv), rhs[k], tp(c.lw[k].t), tp(c.lw[k + 1].rhs),
                          nu, s);
      }
      if (t0 < nlev - 1) {
        std::vector<TailLevelIn> tl(nlev - t0);
        for (int k = t0; k < nlev; ++k) {
          TailLevelIn& e = tl[k - t0];
          const LevelView<float> v = view<float>(c, k);
          e.op = v.ch;
          e.dinv = reinterpret_cast<const float*>(tp(c.lw[k].dinv));
          e.rhs = reinterpret_cast<const float*>(rhs[k]);
          e.z = reinterpret_cast<float*>(zz[k]);
        }
        launch_vtail(tl.data(), nlev - t0, c.kinv.p, (int)c.lev[nlev - 1].n, B, s);
      } else {
        launch_coarse_solve<T>((int)c.lev[nlev - 1].n, B, c.kinv.p, rhs[nlev - 1], zz[nlev - 1], s);
      }
      for (int k = t0 - 1; k >= 0; --k) {
        int g;
        if (k == 0 && fine1)
          g = launch_vfine_up(view<float>(c, 0), B, reinterpret_cast<const float*>(lam2T()), c.prm.smoother,
                              c.prm.omega, reinterpret_cast<const float*>(rhs[0]),
                              reinterpret_cast<const float*>(zz[1]), reinterpret_cast<float*>(zz[0]), part, s);
        else
          g = launch_vup<T>(view<T>(c, k), B, lam2T(), tp(c.lw[k].dinv), rhs[k], zz[k + 1], tp(c.lw[k].t), zz[k],
                            k == 0 ? part : nullptr, nu, s);
        if (k == 0) nb = g;
      }
      return nb;
    }
    for (int k = 0; k < nlev - 1; ++k) {
      LevelView<T> L = view<T>(c, k);
      const T* dinv = tp(c.lw[k].dinv);
      launch_smooth_zero<T>(L, B, lam2T(), dinv, rhs[k], zz[k], nu >= 2 ? 1 : 0, c.maxblk, s);
      sweeps(k, nu - std::min(nu, 2), rhs[k], zz[k], tp(c.lw[k].t), nullptr, nullptr);
      launch_residual<T>(L, B, lam2T(), rhs[k], zz[k], tp(c.lw[k].res), c.maxblk, s);
      launch_restrict<T>(c.lev[k + 1].nv, c.lev[k + 1].nh, B, tp(c.lw[k].res), tp(c.lw[k + 1].rhs), c.maxblk, s);
    }
    launch_coarse_solve<T>((int)c.lev[nlev - 1].n, B, c.kinv.p, rhs[nlev - 1], zz[nlev - 1], s);
    for (int k = nlev - 2; k >= 0; --k) {
      launch_prolong_add<T>(c.lev[k + 1].nv, c.lev[k + 1].nh, B, zz[k + 1], zz[k], c.maxblk, s);
      sweeps(k, nu, rhs[k], zz[k], tp(c.lw[k].t), k == 0 ? part : nullptr, k == 0 ? &nb : nullptr);
    }
    return nb;
  }

  // ---- setup of one batch --------------------------------------------
  void setup(const std::vector<double>& lam) {
    std::vector<double> l2(B);
    std::vector<T> l2t(B);
    for (int j = 0; j < B; ++j) { l2[j] = lam[j] * lam[j]; l2t[j] = (T)l2[j]; }
    LCMG_CUDA(cudaMemcpyAsync(c.lam2.p, l2.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
    LCMG_CUDA(cudaMemcpyAsync(c.lam2T.p, l2t.data(), sizeof(T) * B, cudaMemcpyHostToDevice, s));
    // FP16 smoother data: every column at one lambda, the two-kernels-per-
    // level cycle, mixed precision; the coarse rows of K(lambda) per lambda
    bool one_lam = true;
    for (int j = 1; j < B; ++j) one_lam = one_lam && lam[j] == lam[0];
    c.h16_on = false;
    if (std::is_same<T, float>::value && c.prm.smoother_fp16 && one_lam && !c.prm.autotune && vf_on()) {
      for (int k = 1; k < nlev; ++k) {
        Level& g = c.lev[k];
        g.hscale = half_scale(l2[0] * g.glmax + g.gamax);
        const int gg = (int)std::min<int64_t>((kCompactOff * g.n + kBlock - 1) / kBlock, c.maxblk);
        klaunch(k_compact_rows, dim3(gg), dim3(kBlock), 0, s, g.n, (const double*)g.gl.p, (const double*)g.ga.p,
                l2[0], g.hscale, g.hrows.p);
        LCMG_LAUNCHED();
      }
      c.h16_on = true;
    }
    for (int k = 0; k < nlev; ++k)
      launch_dinv<T>(view<T>(c, k), B, c.lam2.p, c.prm.smoother, c.prm.omega, tp(c.lw[k].dinv), c.maxblk, s);
    launch_dense_setup(view<double>(c, nlev - 1), B, c.lam2.p, c.Mw.p, c.Ww.p, c.kinv.p, c.s_info.p, c.maxblk, s);
    // the host copy of lam2 must stay valid until the copies complete
    LCMG_CUDA(cudaStreamSynchronize(s));
    std::vector<int> info(B);
    copy_sync(c.stream, info.data(), c.s_info.p, sizeof(int) * B, cudaMemcpyDeviceToHost);
    for (int j = 0; j < B; ++j)
      if (info[j] != 0) throw ArgError("coarsest-level Cholesky failed (pivot " + std::to_string(info[j]) + ")");
  }

  void read_counters() {
    LCMG_CUDA(cudaMemcpyAsync(c.h_counters, c.s_counters.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    LCMG_CUDA(cudaStreamSynchronize(s));
  }

  // one PCG iteration for all active columns
  void iterate_once(bool time_it = false) {
    timing_now = time_it;
    ColState st = colstate(c);
    T* P = tp(c.p);
    T* Q = tp(c.q);
    T* R = tp(c.r);
    T* Z = tp(c.z);
    // mixed path: a reliable update once ||r|| has fallen 100x since the last
    // one (each costs two FP64 operator passes; at 10x the 2048^2 chain
    // spent 2.4% more time for the same iteration counts).  Convergence is
    // always decided on the FP64 true residual.
    const double trig = std::is_same<T, float>::value ? 1e-4 : 0.0;
    const int nb_pq = apply_K(P, Q, c.part_pq.p);
    T* X = std::is_same<T, double>::value ? reinterpret_cast<T*>(c.x64.p) : reinterpret_cast<T*>(c.xlo.p);
    int nb_rr;
    const bool alpha_fused = B == 1 && c.prm.alpha_fuse;
    if (alpha_fused) {  // alpha inside the update
      nb_rr = launch_update_xr_alpha<T, T>(c.n, st, nb_pq, c.part_pq.p, P, Q, X, R, c.part_rr.p, c.maxblk, s);
    } else {
      klaunch(k_scalar_col_alpha, dim3(B), dim3(kColThreads), 0, s, B, nb_pq, c.part_pq.p, st);
      LCMG_LAUNCHED();
      nb_rr = launch_update_xr<T, T>(c.n, B, st, P, Q, X, R, c.part_rr.p, c.maxblk, s);
    }
    mark();
    const int nb_rz = vcycle(R, Z, c.part_rz.p);
    mark();
    if (alpha_fused && c.prm.beta_fuse && !c.prm.keep_direction) {  // beta inside the p update
      launch_update_p_beta<T>(c.n, st, nb_rr, c.part_rr.p, nb_rz, c.part_rz.p, c.prm.maxit, trig, Z, P, c.maxblk, s);
      return;
    }
    klaunch(k_scalar_col_beta, dim3(B), dim3(kColThreads), 0, s, B, nb_rr, c.part_rr.p, nb_rz, c.part_rz.p, st,
            c.prm.maxit, trig);
    LCMG_LAUNCHED();
    launch_update_p<T>(c.n, B, st, Z, P, c.maxblk, s);
  }

  // true-residual check of pending columns; on the mixed path also the
  // reliable update of every running column
  void true_check(bool replace_active) {
    ColState st = colstate(c);
    if (!std::is_same<T, double>::value) {
      const int g = (int)std::min<int64_t>(((int64_t)c.n * B + kBlock - 1) / kBlock, c.maxblk);
      klaunch(k_flush_x, dim3(g), dim3(kBlock), 0, s, (int64_t)c.n * B, c.xlo.p, c.x64.p);
      LCMG_LAUNCHED();
    }
    const int nb = true_residual(c.part_x.p);
    klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, s, B, nb, c.part_x.p, c.s_rrtrue.p);
    LCMG_LAUNCHED();
    klaunch(k_true_check, dim3(1), dim3(kBlock), 0, s, B, c.s_rrtrue.p, st, replace_active ? 1 : 0, c.s_flag.p);
    LCMG_LAUNCHED();
    const int g = grid_for(c.n, B, c.maxblk);
    klaunch(k_take_residual<T>, dim3(g), dim3(kBlock), 0, s, c.n, B, c.s_flag.p, c.r64.p, tp(c.r));
    LCMG_LAUNCHED();
    read_counters();
    if (c.h_counters[3] > 0) {  // restarted columns: z = B r, p = z, rz = r.z
      const int nbz = vcycle(tp(c.r), tp(c.z), c.part_rz.p);
      klaunch(k_restart_finish<T>, dim3(g), dim3(kBlock), 0, s, c.n, B, nbz, c.part_rz.p, c.s_flag.p, st, tp(c.z), tp(c.p));
      LCMG_LAUNCHED();
    }
  }

  // Autotuner (params.autotune): on the first batch of width B, time the
  // one-column SpMV configurations of each operator pass and both V-cycle
  // forms on this context's operator and hierarchy (CUDA events, 3 runs
  // after one warm-up, on scratch vectors), keep the fastest per width.
  void autotune() {
    if (!c.prm.autotune || c.tuned.count(tune_key())) return;
    Tuned t;
    LCMG_CUDA(cudaMemsetAsync(c.p.p, 0, sizeof(T) * c.n * B, s));
    LCMG_CUDA(cudaMemsetAsync(c.r.p, 0, sizeof(T) * c.n * B, s));
    cudaEvent_t e0, e1;
    LCMG_CUDA(cudaEventCreate(&e0));
    LCMG_CUDA(cudaEventCreate(&e1));
    auto time = [&](auto&& fn) {
      fn();
      LCMG_CUDA(cudaEventRecord(e0, s));
      for (int i = 0; i < 3; ++i) fn();
      LCMG_CUDA(cudaEventRecord(e1, s));
      LCMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      LCMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return ms;
    };
    auto apply = [&] { apply_K(tp(c.p), tp(c.q), c.part_pq.p); };
    if (c.fwd == 1 && B == 1) {
      // transposed pass at its default while A's configurations are timed,
      // then A at its winner while the transposed pass's are timed
      float best = 1e30f;
      for (int v = 1; v <= 3; ++v) {
        var_a = v;
        const float ms = time(apply);
        if (ms < best) { best = ms; t.var_a = v; }
      }
      var_a = t.var_a;
      best = 1e30f;
      for (int v = 1; v <= 6; ++v) {
        var_at = v;
        const float ms = time(apply);
        if (ms < best) { best = ms; t.var_at = v; }
      }
      var_at = t.var_at;
    }
    const int nu = c.prm.nu;
    if (nlev >= 2 && (nu == 1 || nu == 2)) {
      float best = 1e30f;
      for (int f = 0; f <= 1; ++f) {
        vf_force = f;
        const float ms = time([&] { vcycle(tp(c.r), tp(c.z), c.part_rz.p); });
        if (ms < best) { best = ms; t.vfuse = f; }
      }
      vf_force = t.vfuse;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.tuned[tune_key()] = t;
  }

  // Run PCG on the batch whose x64 (initial guesses) and c64 (right-hand
  // sides A^T b) are set.  Returns the number of batch iterations.
  int64_t run(const std::vector<double>& lam) {
    setup(lam);
    autotune();
    c.stats.tuned_spmv_a = var_a;
    c.stats.tuned_spmv_at = var_at;
    c.stats.tuned_vfuse = vf_force;
    ColState st = colstate(c);
    // ||c||^2 and the true initial residual
    const int g = grid_for(c.n, B, c.maxblk);
    klaunch(k_col_dot<double>, dim3(g), dim3(kBlock), 0, s, c.n, B, c.c64.p, c.c64.p, c.part_x.p);
    LCMG_LAUNCHED();
    klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, s, B, g, c.part_x.p, c.s_cc.p);
    LCMG_LAUNCHED();
    klaunch(k_zero_cols, dim3(g), dim3(kBlock), 0, s, c.n, B, c.s_cc.p, c.x64.p);
    LCMG_LAUNCHED();
    const int nb = true_residual(c.part_x.p);
    klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, s, B, nb, c.part_x.p, c.s_rrtrue.p);
    LCMG_LAUNCHED();
    klaunch(k_init_state, dim3(1), dim3(kBlock), 0, s, B, c.prm.tol, c.s_cc.p, c.s_rrtrue.p, st);
    LCMG_LAUNCHED();
    // r = (T) r64 for every column
    LCMG_CUDA(cudaMemsetAsync(c.s_flag.p, 0, sizeof(int) * B, s));
    {
      std::vector<int> ones(B, 1);
      LCMG_CUDA(cudaMemcpyAsync(c.s_flag.p, ones.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
      klaunch(k_take_residual<T>, dim3(g), dim3(kBlock), 0, s, c.n, B, c.s_flag.p, c.r64.p, tp(c.r));
      LCMG_LAUNCHED();
      LCMG_CUDA(cudaStreamSynchronize(s));
    }
    if (!std::is_same<T, double>::value) LCMG_CUDA(cudaMemsetAsync(c.xlo.p, 0, sizeof(float) * c.n * B, s));
    // z = B r ; p = z ; rz = r.z   (for every column; frozen ones are unaffected)
    const int nbz = vcycle(tp(c.r), tp(c.z), c.part_rz.p);
    klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, s, B, nbz, c.part_rz.p, c.s_rz.p);
    LCMG_LAUNCHED();
    LCMG_CUDA(cudaMemcpyAsync(c.s_rz2.p, c.s_rz.p, sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
    launch_copy_cols<T>(c.n, B, nullptr, tp(c.z), tp(c.p), c.maxblk, s);
    int64_t batch_its = 0;
    cudaEvent_t e0, e1;
    LCMG_CUDA(cudaEventCreate(&e0));
    LCMG_CUDA(cudaEventCreate(&e1));
    LCMG_CUDA(cudaEventRecord(e0, s));
    // counters as left by k_init_state are not set: read active directly
    std::vector<int> act(B);
    LCMG_CUDA(cudaMemcpyAsync(act.data(), c.s_active.p, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
    LCMG_CUDA(cudaStreamSynchronize(s));
    int active = 0;
    for (int v : act) active += v;
    const int every = c.prm.check_every;
    const bool mixed = !std::is_same<T, double>::value;
    // one block of `every` iterations, captured once into a CUDA graph
    cudaGraphExec_t exec = nullptr;
    int64_t per_block = 0;  // kernels in one captured block
    c.tev_used = 0;
    if (c.prm.graphs && active > 0) {
      cudaGraph_t graph = nullptr;
      const int64_t l0 = launch_counter();
      LCMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      try {
        for (int i = 0; i < every; ++i) iterate_once(i == 0);
      } catch (...) {
        cudaStreamEndCapture(s, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      per_block = launch_counter() - l0;
      launch_counter() = l0;  // captured, not executed
      LCMG_CUDA(cudaStreamEndCapture(s, &graph));
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      LCMG_CUDA(ie);
    }
    struct ExecGuard {
      cudaGraphExec_t e;
      ~ExecGuard() {
        if (e) cudaGraphExecDestroy(e);
      }
    } guard{exec};
    while (active > 0) {
      if (exec) {
        LCMG_CUDA(cudaGraphLaunch(exec, s));
        launch_counter() += per_block;
      } else {
        c.tev_used = 0;
        for (int i = 0; i < every; ++i) iterate_once(i == 0);
      }
      batch_its += every;
      read_counters();
      collect_timing();
      active = c.h_counters[0];
      const int pending = c.h_counters[1];
      const int votes = c.h_counters[2];
      if (pending > 0 || (mixed && votes > 0) || active == 0) {
        true_check(mixed);
        active = c.h_counters[0];
      }
      if (batch_its > (int64_t)c.prm.maxit + 4LL * every + 64) break;  // safety net
    }
    if (!std::is_same<T, double>::value) {
      const int gg = (int)std::min<int64_t>(((int64_t)c.n * B + kBlock - 1) / kBlock, c.maxblk);
      klaunch(k_flush_x, dim3(gg), dim3(kBlock), 0, s, (int64_t)c.n * B, c.xlo.p, c.x64.p);
      LCMG_LAUNCHED();
    }
    LCMG_CUDA(cudaEventRecord(e1, s));
    LCMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.stats.iterate_ms += ms;
    c.stats.batch_iterations += batch_its;
    return batch_its;
  }
};

template <class T>
const T* Batch<T>::psfT() {
  return std::is_same<T, double>::value ? reinterpret_cast<const T*>(c.psf64.p)
                                        : reinterpret_cast<const T*>(c.psf32.p);
}

// Algorithmic (compulsory) DRAM bytes of the two operator passes for a
// batch of B columns in precision T: the operator data once, every input
// vector read once and every output written once.
template <class T>
static void op_bytes(const lcmg_ctx& c, int B, int64_t* first, int64_t* second) {
  const int64_t sT = sizeof(T), sB = B;
  if (c.fwd == 1) {
    const int64_t sV = (std::is_same<T, float>::value || c.vdtype == 0) ? 4 : 8;
    // the one-column transposed pass reads 16-bit column offsets and a base per row
    const bool c16 = B == 1 && c.c16_ok && c.prm.compact_cols;
    *first = c.nnz * (sV + 4) + (c.m + 1) * 8 + c.n * sB * sT + c.m * sB * sT;
    *second = c.nnz * (sV + (c16 ? 2 : 4)) + (c.n + 1) * 8 + (c16 ? c.n * 4 : 0) + c.m * sB * sT +
              2 * c.n * sB * sT + 2 * c.n * sT + c.n * sB * sT;
  } else {
    *first = 2 * c.n * sB * sT;
    *second = 3 * c.n * sB * sT + 2 * c.n * sT;
  }
}

template <class T>
int Batch<T>::apply_K(const T* P, T* Q, double* part) {
  T* Y = tp(c.y);
  mark();
  int nb;
  if (c.fwd == 1) {
    SpmmArgs a = args(false, B);
    SpmmArgs at = args(true, B);
    a.variant = var_a;
    at.variant = var_at;
    if (std::is_same<T, float>::value) {
      launch_spmm<float, float, float, 0>(a, c.v32.p, reinterpret_cast<const float*>(P), reinterpret_cast<float*>(Y),
                                          view<float>(c, 0).fine_op(), nullptr, nullptr, nullptr, nullptr,
                                          nullptr, c.maxblk, s);
      mark();
      nb = launch_spmm<float, float, float, 1>(at, c.vT32.p, reinterpret_cast<const float*>(Y),
                                               reinterpret_cast<float*>(Q), view<float>(c, 0).fine_op(),
                                               reinterpret_cast<const float*>(P), nullptr, c.lam2.p, nullptr,
                                               part, c.maxblk, s);
    } else {
      const double* Pd = reinterpret_cast<const double*>(P);
      double* Qd = reinterpret_cast<double*>(Q);
      double* Yd = reinterpret_cast<double*>(Y);
      if (c.vdtype == 1) {
        launch_spmm<double, double, double, 0>(a, c.v64.p, Pd, Yd, fop64(), nullptr, nullptr, nullptr, nullptr,
                                               nullptr, c.maxblk, s);
        mark();
        nb = launch_spmm<double, double, double, 1>(at, c.vT64.p, Yd, Qd, fop64(), Pd, nullptr, c.lam2.p,
                                                    nullptr, part, c.maxblk, s);
      } else {
        launch_spmm<float, double, double, 0>(a, c.v32.p, Pd, Yd, fop64(), nullptr, nullptr, nullptr, nullptr,
                                              nullptr, c.maxblk, s);
        mark();
        nb = launch_spmm<float, double, double, 1>(at, c.vT32.p, Yd, Qd, fop64(), Pd, nullptr, c.lam2.p,
                                                   nullptr, part, c.maxblk, s);
      }
    }
  } else if (c.sep) {
    // separable PSF: u = (I (x) T_v) p, then q = (T_h (x) I) u + lam^2 L^T W L p with p.q
    launch_band<T, T, 0, BAND_STORE>(c.nv, c.nh, B, band_vt(), P, Y, fop(), nullptr, nullptr, nullptr, nullptr,
                                     nullptr, c.maxblk, s);
    mark();
    nb = launch_band<T, T, 1, BAND_NORMAL>(c.nv, c.nh, B, band_ht(), Y, Q, fop(), P, nullptr, c.lam2.p, nullptr,
                                           part, c.maxblk, s);
  } else {
    // PSF operator
    nb = grid_for(c.n, B, c.maxblk);
    PsfArgs pa = psf();
    klaunch(k_psf_forward<T, 0>, dim3(nb), dim3(kBlock), 0, s, pa, psfT(), B, P, Y, nullptr, 1, 1, nullptr);
    LCMG_LAUNCHED();
    mark();
    klaunch(k_psf_normal<T, T, 1>, dim3(nb), dim3(kBlock), 0, s, pa, psfT(), B, Y, fop(), P, nullptr, c.lam2.p, Q, part);
    LCMG_LAUNCHED();
  }
  mark();
  return nb;
}

template <class T>
int Batch<T>::true_residual(double* part) {
  double* Y = c.y64.p;
  if (c.fwd == 1) {
    SpmmArgs a = args(false, B);
    SpmmArgs at = args(true, B);
    if (c.vdtype == 1) {
      launch_spmm<double, double, double, 0>(a, c.v64.p, c.x64.p, Y, fop64(), nullptr, nullptr, nullptr, nullptr,
                                             nullptr, c.maxblk, s);
      return launch_spmm<double, double, double, 3>(at, c.vT64.p, Y, c.r64.p, fop64(), c.x64.p, c.c64.p,
                                                    c.lam2.p, nullptr, part, c.maxblk, s);
    }
    launch_spmm<float, double, double, 0>(a, c.v32.p, c.x64.p, Y, fop64(), nullptr, nullptr, nullptr, nullptr,
                                          nullptr, c.maxblk, s);
    return launch_spmm<float, double, double, 3>(at, c.vT32.p, Y, c.r64.p, fop64(), c.x64.p, c.c64.p, c.lam2.p,
                                                 nullptr, part, c.maxblk, s);
  }
  if (c.sep) {
    Band<double> bv = make_band<double>(c.sp_vt, c.sep_dv64.p), bh = make_band<double>(c.sp_ht, c.sep_dh64.p);
    launch_band<double, double, 0, BAND_STORE>(c.nv, c.nh, B, bv, c.x64.p, Y, fop64(), nullptr, nullptr, nullptr,
                                               nullptr, nullptr, c.maxblk, s);
    return launch_band<double, double, 1, BAND_TRUERES>(c.nv, c.nh, B, bh, Y, c.r64.p, fop64(), c.x64.p, c.c64.p,
                                                        c.lam2.p, nullptr, part, c.maxblk, s);
  }
  const int g = grid_for(c.n, B, c.maxblk);
  PsfArgs pa = psf();
  klaunch(k_psf_forward<double, 0>, dim3(g), dim3(kBlock), 0, s, pa, c.psf64.p, B, c.x64.p, Y, nullptr, 1, 1, nullptr);
  LCMG_LAUNCHED();
  klaunch(k_psf_normal<double, double, 3>, dim3(g), dim3(kBlock), 0, s, pa, c.psf64.p, B, Y, fop64(), c.x64.p, c.c64.p, c.lam2.p,
                                                       c.r64.p, part);
  LCMG_LAUNCHED();
  return g;
}

// ---------------------------------------------------------------------------
// Solve driver
// ---------------------------------------------------------------------------
// c = A^T b for the nrhs right-hand sides (b interleaved [m][nrhs] in c.bvec)
static void compute_rhs(lcmg_ctx& c, int nrhs) {
  double* cv = c.cvec.need((size_t)c.n * nrhs);
  if (c.fwd == 1) {
    SpmmArgs a = csr_args(c, true, nrhs);
    FineOp<double> f = view<double>(c, 0).fine_op();
    if (c.vdtype == 1)
      launch_spmm<double, double, double, 0>(a, c.vT64.p, c.bvec.p, cv, f, nullptr, nullptr, nullptr, nullptr,
                                             nullptr, c.maxblk, c.stream);
    else
      launch_spmm<float, double, double, 0>(a, c.vT32.p, c.bvec.p, cv, f, nullptr, nullptr, nullptr, nullptr,
                                            nullptr, c.maxblk, c.stream);
  } else if (c.sep) {
    // A^T b = (A_h^T (x) A_v^T) b: the flipped 1-D correlations along i, then j
    double* tmp = c.sep_tmp.need((size_t)c.n * nrhs);
    FineOp<double> f = view<double>(c, 0).fine_op();
    launch_band<double, double, 0, BAND_STORE>(c.nv, c.nh, nrhs, make_band<double>(c.sp_vat, nullptr), c.bvec.p, tmp,
                                               f, nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, c.stream);
    launch_band<double, double, 1, BAND_STORE>(c.nv, c.nh, nrhs, make_band<double>(c.sp_hat, nullptr), tmp, cv, f,
                                               nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, c.stream);
  } else {
    PsfArgs pa{};
    pa.nv = c.nv; pa.nh = c.nh; pa.rv = c.rv; pa.rh = c.rh; pa.psf = c.psf64.p;
    klaunch(k_psf_rhs, dim3(grid_for(c.n, nrhs, c.maxblk)), dim3(kBlock), 0, c.stream, pa, nrhs, c.bvec.p, cv);
    LCMG_LAUNCHED();
  }
}

// ---------------------------------------------------------------------------
// The paper's own preconditioner and Krylov method (params.precond = 1,
// Sec. 3.2-3.3): multigrid on the whole normal operator with the one-sided
// coarse operators A_{k+1} = A_k P_k (M_k^T M_k is the Galerkin stencil
// G_L^k already held for the default preconditioner), V(2,1) with
// Jacobi-preconditioned CG relaxation, an exact coarsest solve of
// A_c^T A_c + lam^2 G_L^c, and right-preconditioned flexible GMRES.  FP64,
// one column at a time (the paper's lambda chain).
// ---------------------------------------------------------------------------
constexpr int kPmNu1 = 2, kPmNu2 = 1;  // CG relaxation steps before / after the coarse correction


// weight of coarse cell I in the cell-centred linear interpolation to fine
// cell a (nc coarse cells; an outside neighbour's weight goes to the parent)
static double interp_w(int a, int I, int nc) {
  const int d = a - 2 * I;
  if (d == 0) return I == 0 ? 1.0 : 0.75;
  if (d == 1) return I == nc - 1 ? 1.0 : 0.75;
  if (d == -1 || d == 2) return 0.25;
  return 0.0;
}

// A P for P = P_h (x) P_v from the nv/2 x nh/2 grid to the nv x nh grid,
// by the threaded host product with the explicit P (a fine pixel's row
// holds w_j * w_i for its 2 x 2 coarse parents): every nonzero of A adds to
// a coarse column at most once, in the order of A's nonzeros, whatever the
// thread count
static HostCsr times_p(const HostCsr& A, int nv, int nh) {
  const int nvc = nv / 2, nhc = nh / 2;
  HostCsr P;
  P.rows = (int64_t)nv * nh;
  P.cols = (int64_t)nvc * nhc;
  P.rp.assign(P.rows + 1, 0);
  for (int j = 0; j < nh; ++j)
    for (int i = 0; i < nv; ++i) {
      const int Is[2] = {i >> 1, (i & 1) ? (i >> 1) + 1 : (i >> 1) - 1};
      const int Js[2] = {j >> 1, (j & 1) ? (j >> 1) + 1 : (j >> 1) - 1};
      for (int u = 0; u < 2; ++u) {
        const int J = Js[u];
        if (J < 0 || J >= nhc) continue;
        const double wj = interp_w(j, J, nhc);
        for (int t = 0; t < 2; ++t) {
          const int I = Is[t];
          if (I < 0 || I >= nvc) continue;
          P.ci.push_back(I + J * nvc);
          P.v.push_back(wj * interp_w(i, I, nvc));
        }
      }
      P.rp[(int64_t)i + (int64_t)j * nv + 1] = (int64_t)P.ci.size();
    }
  return amg::spgemm(A, P);
}

// host copy of the CSR forward operator A (values in FP64)
static HostCsr host_forward(lcmg_ctx& c) {
  cudaStream_t s = c.stream;
  HostCsr A;
  A.rows = c.m;
  A.cols = c.n;
  A.rp.resize(c.m + 1);
  A.ci.resize(c.nnz);
  A.v.resize(c.nnz);
  copy_sync(s, A.rp.data(), c.rp.p, sizeof(int64_t) * (c.m + 1), cudaMemcpyDeviceToHost);
  copy_sync(s, A.ci.data(), c.ci.p, sizeof(int32_t) * c.nnz, cudaMemcpyDeviceToHost);
  if (c.vdtype == 1) {
    copy_sync(s, A.v.data(), c.v64.p, sizeof(double) * c.nnz, cudaMemcpyDeviceToHost);
  } else {
    std::vector<float> vf(c.nnz);
    copy_sync(s, vf.data(), c.v32.p, sizeof(float) * c.nnz, cudaMemcpyDeviceToHost);
    for (int64_t k = 0; k < c.nnz; ++k) A.v[k] = vf[k];
  }
  return A;
}

// upload the one-sided A_k (k >= 1, n_k columns) with its transpose and
// diag(A_k^T A_k); on the coarsest level also the dense A_c^T A_c
static void upload_one_sided(lcmg_ctx& c, int k, const HostCsr& A, bool coarsest) {
  cudaStream_t s = c.stream;
  HostCsr T = amg::transpose(A);
  PmLevel& P = c.pm[k];
  P.nnz = (int64_t)A.ci.size();
  copy_sync(s, P.rp.need(A.rows + 1 + kCsrPad), A.rp.data(), sizeof(int64_t) * (A.rows + 1), cudaMemcpyHostToDevice);
  copy_sync(s, P.ci.need(P.nnz + kCsrPad), A.ci.data(), sizeof(int32_t) * P.nnz, cudaMemcpyHostToDevice);
  copy_sync(s, P.v.need(P.nnz + kCsrPad), A.v.data(), sizeof(double) * P.nnz, cudaMemcpyHostToDevice);
  copy_sync(s, P.rpT.need(T.rows + 1 + kCsrPad), T.rp.data(), sizeof(int64_t) * (T.rows + 1), cudaMemcpyHostToDevice);
  copy_sync(s, P.ciT.need(P.nnz + kCsrPad), T.ci.data(), sizeof(int32_t) * P.nnz, cudaMemcpyHostToDevice);
  copy_sync(s, P.vT.need(P.nnz + kCsrPad), T.v.data(), sizeof(double) * P.nnz, cudaMemcpyHostToDevice);
  const int64_t nk = A.cols;
  const int g = (int)std::min<int64_t>((nk * 32 + kBlock - 1) / kBlock, c.maxblk);
  klaunch(k_diag_ata<double>, dim3(g), dim3(kBlock), 0, s, nk, P.rpT.p, P.vT.p, P.dA.need(nk));
  LCMG_LAUNCHED();
  if (coarsest) {  // dense A_c^T A_c, rows of A_c in order
    const int64_t nc = nk;
    std::vector<double> AtA((size_t)nc * nc, 0.0);
    for (int64_t r = 0; r < A.rows; ++r)
      for (int64_t a = A.rp[r]; a < A.rp[r + 1]; ++a)
        for (int64_t b2 = A.rp[r]; b2 < A.rp[r + 1]; ++b2)
          AtA[(size_t)A.ci[a] * nc + A.ci[b2]] += A.v[a] * A.v[b2];
    copy_sync(s, c.pm_AtAc.need(nc * nc), AtA.data(), sizeof(double) * nc * nc, cudaMemcpyHostToDevice);
  }
}

static void alloc_pm_work(lcmg_ctx& c, const std::vector<int64_t>& sizes) {
  const int L = (int)sizes.size();
  c.pmw.clear();
  c.pmw.resize(L);
  for (int k = 0; k < L; ++k) {
    PmWork& W = c.pmw[k];
    const int64_t nk = sizes[k];
    W.b.need(nk); W.x.need(nk);
    if (k + 1 < L) {
      for (auto* b : {&W.r, &W.z, &W.p, &W.q, &W.t, &W.dinv}) b->need(nk);
      W.y.need(c.m);
      for (auto* b : {&W.pa, &W.pb, &W.ppq}) b->need(kMaxBlocks);
    }
  }
  const size_t nc = (size_t)sizes[L - 1];
  c.kinv.need(nc * nc); c.Mw.need(nc * nc); c.Ww.need(nc * nc);
}

template <class I>
static I* upload(cudaStream_t s, DevBuf<I>& buf, const std::vector<I>& h, size_t pad = 0) {
  I* d = buf.need(h.size() + pad);
  copy_sync(s, d, h.data(), sizeof(I) * h.size(), cudaMemcpyHostToDevice);
  return d;
}

// The paper's hierarchy with classical AMG (Sec. 3.1-3.2): coarsen
// G_L = L^T D^2 L on the host, then A_{k+1} = A_k P_k; rebuilt per D.
static void pm_build_amg(lcmg_ctx& c) {
  if (c.am_ok) return;
  if (c.fwd != 1) throw ArgError("the paper's preconditioner needs a CSR forward operator");
  cudaStream_t s = c.stream;
  std::vector<double> d(c.ne);
  copy_sync(s, d.data(), c.d.p, sizeof(double) * c.ne, cudaMemcpyDeviceToHost);
  const HostCsr K0 = amg::weighted_laplacian(c.nv, c.nh, d.data());
  const int maxlev = c.prm.levels > 0 ? c.prm.levels : 64;
  amg::Hierarchy H = amg::hierarchy(K0, maxlev, c.prm.amg_coarse_max, amg::kTheta, c.prm.coarsening == 2, s);
  const int L = (int)H.K.size();
  if (L < 2) throw ArgError("classical AMG made no coarse level (grid at most amg_coarse_max points, or levels = 1)");
  const int64_t nc = H.K[L - 1].rows;
  if (nc > 2048)
    throw ArgError("the coarsest classical AMG level has " + std::to_string(nc) +
                   " points (more than 2048): allow more levels");
  c.am.clear();
  c.am.resize(L);
  std::vector<int64_t> sizes(L);
  for (int k = 0; k < L; ++k) {
    AmLevel& a = c.am[k];
    a.n = sizes[k] = H.K[k].rows;
    if (k > 0) {
      const HostCsr& G = H.K[k];
      std::vector<double> dg(G.rows, 0.0);
      for (int64_t r = 0; r < G.rows; ++r)
        for (int64_t q = G.rp[r]; q < G.rp[r + 1]; ++q)
          if (G.ci[q] == r) dg[r] = G.v[q];
      upload(s, a.grp, G.rp);
      upload(s, a.gci, G.ci, 1);
      upload(s, a.gv, G.v, 1);
      upload(s, a.gdiag, dg);
    }
    if (k + 1 < L) {
      const HostCsr& P = H.P[k];
      const HostCsr PT = amg::transpose(P);
      upload(s, a.prp, P.rp);
      upload(s, a.pci, P.ci, 1);
      upload(s, a.pv, P.v, 1);
      upload(s, a.ptrp, PT.rp);
      upload(s, a.ptci, PT.ci, 1);
      upload(s, a.ptv, PT.v, 1);
    }
  }
  {  // dense G_L^c
    const HostCsr& G = H.K[L - 1];
    std::vector<double> Gd((size_t)nc * nc, 0.0);
    for (int64_t r = 0; r < G.rows; ++r)
      for (int64_t q = G.rp[r]; q < G.rp[r + 1]; ++q) Gd[(size_t)r * nc + G.ci[q]] = G.v[q];
    upload(s, c.pm_GLc, Gd);
  }
  HostCsr A = host_forward(c);
  c.pm.clear();
  c.pm.resize(L);
  for (int k = 1; k < L; ++k) {
    A = amg::spgemm(A, H.P[k - 1]);
    upload_one_sided(c, k, A, k == L - 1);
  }
  alloc_pm_work(c, sizes);
  LCMG_CUDA(cudaStreamSynchronize(s));
  c.am_ok = true;
  c.pm_levels = 0;  // the geometric one-sided hierarchy is no longer held
}

static void pm_build(lcmg_ctx& c) {
  if (c.prm.coarsening == 1 || c.prm.coarsening == 2) {
    pm_build_amg(c);
    return;
  }
  ensure_hierarchy(c);
  const int L = (int)c.lev.size();
  if (c.pm_levels == L) return;
  if (c.fwd != 1) throw ArgError("the paper's preconditioner needs a CSR forward operator");
  if (L < 2) throw ArgError("the paper's preconditioner needs at least 2 levels");
  cudaStream_t s = c.stream;
  HostCsr A = host_forward(c);
  c.pm.clear();
  c.pm.resize(L);
  for (int k = 1; k < L; ++k) {
    A = times_p(A, c.lev[k - 1].nv, c.lev[k - 1].nh);
    upload_one_sided(c, k, A, k == L - 1);
  }
  std::vector<int64_t> sizes(L);
  for (int k = 0; k < L; ++k) sizes[k] = c.lev[k].n;
  alloc_pm_work(c, sizes);
  LCMG_CUDA(cudaStreamSynchronize(s));
  c.pm_levels = L;
  c.am_ok = false;
}

struct PaperMG {
  lcmg_ctx& c;
  cudaStream_t s;
  bool amg;
  int L;
  explicit PaperMG(lcmg_ctx& c_)
      : c(c_), s(c_.stream), amg(c_.prm.coarsening != 0),
        L(c_.prm.coarsening != 0 ? (int)c_.am.size() : (int)c_.lev.size()) {}

  int64_t nk(int k) const { return amg ? c.am[k].n : c.lev[k].n; }
  int grid(int k) const { return grid_for(nk(k), 1, c.maxblk); }
  GLOp glop(int k) const { return GLOp{c.lev[k].nv, c.lev[k].nh, c.lev[k].n, c.lev[k].gl.p}; }
  CsrGLOp cglop(int k) const {
    const AmLevel& a = c.am[k];
    return CsrGLOp{(int)a.n, a.n, a.grp.p, a.gci.p, a.gv.p, a.gdiag.p};
  }
  FineOp<double> fop() const { return FineOp<double>{c.nv, c.nh, c.ws.p, c.we.p, c.diag.p}; }

  // y = A_k x, t = A_k^T y
  void passes(int k, const double* x, double* y, double* t) {
    const FineOp<double> f = fop();
    if (k == 0) {
      SpmmArgs a = csr_args(c, false, 1), at = csr_args(c, true, 1);
      at.variant = 3;  // the transposed pass in the 8-lane layout, as on the default path
      if (c.vdtype == 1) {
        launch_spmm<double, double, double, 0>(a, c.v64.p, x, y, f, nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, s);
        launch_spmm<double, double, double, 0>(at, c.vT64.p, y, t, f, nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, s);
      } else {
        launch_spmm<float, double, double, 0>(a, c.v32.p, x, y, f, nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, s);
        launch_spmm<float, double, double, 0>(at, c.vT32.p, y, t, f, nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, s);
      }
      return;
    }
    const PmLevel& P = c.pm[k];
    SpmmArgs a{};
    a.rows = c.m; a.rp = P.rp.p; a.ci = P.ci.p; a.B = 1; a.nb = 1; a.nl = 1; a.nrhs = 1;
    SpmmArgs at = a;
    at.rows = nk(k); at.rp = P.rpT.p; at.ci = P.ciT.p;
    launch_spmm<double, double, double, 0>(a, P.v.p, x, y, f, nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, s);
    launch_spmm<double, double, double, 0>(at, P.vT.p, y, t, f, nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, s);
  }
  // MODE 0: q = K_k x with partials of x.q; MODE 1: q = b - K_k x
  template <int MODE>
  void apply(int k, const double* x, const double* b, double* q, double* part) {
    PmWork& W = c.pmw[k];
    passes(k, x, W.y.p, W.t.p);
    const int g = grid(k);
    if (k == 0)
      klaunch(k_pm_lap_add<FineOp<double>, MODE>, dim3(g), dim3(kBlock), 0, s, fop(), nk(0), c.lam2.p, x, W.t.p, b, q, part);
    else if (amg)
      klaunch(k_pm_lap_add<CsrGLOp, MODE>, dim3(g), dim3(kBlock), 0, s, cglop(k), nk(k), c.lam2.p, x, W.t.p, b, q, part);
    else
      klaunch(k_pm_lap_add<GLOp, MODE>, dim3(g), dim3(kBlock), 0, s, glop(k), nk(k), c.lam2.p, x, W.t.p, b, q, part);
    LCMG_LAUNCHED();
  }
  // `steps` CG steps on K_k x = b; zero_x: from x = 0, else from x with r = b - K x
  void relax(int k, const double* b, double* x, int steps, bool zero_x) {
    PmWork& W = c.pmw[k];
    const int64_t n = nk(k);
    const int g = grid(k);
    if (!zero_x) apply<1>(k, x, b, W.r.p, nullptr);
    klaunch(k_pm_cg_init, dim3(g), dim3(kBlock), 0, s, n, zero_x ? 1 : 0, b, W.dinv.p, x, W.r.p, W.z.p, W.p.p, W.pa.p);
    LCMG_LAUNCHED();
    double* cur = W.pa.p;
    double* nxt = W.pb.p;
    for (int st = 0; st < steps; ++st) {
      apply<0>(k, W.p.p, nullptr, W.q.p, W.ppq.p);
      klaunch(k_pm_cg_xr, dim3(g), dim3(kBlock), 0, s, n, cur, g, W.ppq.p, g, W.p.p, W.q.p, W.dinv.p, x, W.r.p,
              W.z.p, nxt);
      LCMG_LAUNCHED();
      if (st + 1 < steps) {
        klaunch(k_pm_cg_p, dim3(g), dim3(kBlock), 0, s, n, nxt, cur, g, W.z.p, W.p.p);
        LCMG_LAUNCHED();
      }
      std::swap(cur, nxt);
    }
  }
  // x = V-cycle(b) on level k (zero initial guess)
  void cycle(int k, const double* b, double* x) {
    if (k == L - 1) {
      launch_coarse_solve<double>((int)nk(k), 1, c.kinv.p, b, x, s);
      return;
    }
    PmWork& W = c.pmw[k];
    PmWork& Wc = c.pmw[k + 1];
    relax(k, b, x, kPmNu1, true);
    apply<1>(k, x, b, W.r.p, nullptr);
    if (amg) {
      const AmLevel& a = c.am[k];
      klaunch(k_pm_csr_mv<false>, dim3(grid(k + 1)), dim3(kBlock), 0, s, nk(k + 1), a.ptrp.p, a.ptci.p, a.ptv.p,
              (const double*)W.r.p, Wc.b.p);
      LCMG_LAUNCHED();
      cycle(k + 1, Wc.b.p, Wc.x.p);
      klaunch(k_pm_csr_mv<true>, dim3(grid(k)), dim3(kBlock), 0, s, nk(k), a.prp.p, a.pci.p, a.pv.p,
              (const double*)Wc.x.p, x);
      LCMG_LAUNCHED();
    } else {
      launch_restrict<double>(c.lev[k + 1].nv, c.lev[k + 1].nh, 1, W.r.p, Wc.b.p, c.maxblk, s);
      cycle(k + 1, Wc.b.p, Wc.x.p);
      launch_prolong_add<double>(c.lev[k + 1].nv, c.lev[k + 1].nh, 1, Wc.x.p, x, c.maxblk, s);
    }
    relax(k, b, x, kPmNu2, false);
  }
  // per lambda: Jacobi diagonals and the coarsest factorisation
  void setup(double lam) {
    const double l2 = lam * lam;
    copy_sync(s, c.lam2.p, &l2, sizeof(double), cudaMemcpyHostToDevice);
    for (int k = 0; k + 1 < L; ++k) {
      const int g = grid(k);
      const double* dA = k == 0 ? c.diag.p : c.pm[k].dA.p;
      if (k == 0)
        klaunch(k_pm_dinv<FineOp<double>>, dim3(g), dim3(kBlock), 0, s, fop(), nk(0), c.lam2.p, dA, c.pmw[0].dinv.p);
      else if (amg)
        klaunch(k_pm_dinv<CsrGLOp>, dim3(g), dim3(kBlock), 0, s, cglop(k), nk(k), c.lam2.p, dA, c.pmw[k].dinv.p);
      else
        klaunch(k_pm_dinv<GLOp>, dim3(g), dim3(kBlock), 0, s, glop(k), nk(k), c.lam2.p, dA, c.pmw[k].dinv.p);
      LCMG_LAUNCHED();
    }
    const int64_t nc = nk(L - 1);
    const int gd = (int)std::min<int64_t>((nc * nc + kBlock - 1) / kBlock, c.maxblk);
    if (amg)
      klaunch(k_pm_dense_add, dim3(gd), dim3(kBlock), 0, s, nc * nc, c.lam2.p, c.pm_AtAc.p, c.pm_GLc.p, c.Mw.p);
    else
      klaunch(k_pm_dense, dim3(gd), dim3(kBlock), 0, s, glop(L - 1), c.lam2.p, c.pm_AtAc.p, c.Mw.p);
    LCMG_LAUNCHED();
    klaunch(k_cholesky_inverse, dim3(1), dim3(kBlock), 0, s, (int)nc, c.Mw.p, c.Ww.p, c.kinv.p, c.s_info.p);
    LCMG_LAUNCHED();
    int info = 0;
    copy_sync(s, &info, c.s_info.p, sizeof(int), cudaMemcpyDeviceToHost);
    if (info != 0) throw ArgError("coarsest-level Cholesky failed (pivot " + std::to_string(info) + ")");
  }
  double dot(const double* a, const double* b) {
    const int g = grid_for(c.n, 1, c.maxblk);
    klaunch(k_col_dot<double>, dim3(g), dim3(kBlock), 0, s, c.n, 1, a, b, c.part_x.p);
    LCMG_LAUNCHED();
    klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, s, 1, g, c.part_x.p, c.s_out.p);
    LCMG_LAUNCHED();
    double v = 0.0;
    copy_sync(s, &v, c.s_out.p, sizeof(double), cudaMemcpyDeviceToHost);
    return v;
  }
  // h[0 .. cnt) = V[0 .. cnt)^T w, then w -= V h (one classical Gram-Schmidt pass)
  void cgs_pass(int cnt, double* w, double* h) {
    const int64_t n = c.n;
    const int nbd = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, 128);
    klaunch(k_pm_multidot, dim3(nbd, cnt), dim3(kBlock), 0, s, n, cnt, c.pm_V.p, n, w, c.pm_part.p);
    LCMG_LAUNCHED();
    klaunch(k_pm_sum_rows, dim3((cnt + kBlock / 32 - 1) / (kBlock / 32)), dim3(kBlock), 0, s, cnt, nbd, c.pm_part.p, h, 0);
    LCMG_LAUNCHED();
    klaunch(k_pm_orth, dim3(grid_for(n, 1, c.maxblk)), dim3(kBlock), 0, s, n, cnt, c.pm_V.p, n, h, w);
    LCMG_LAUNCHED();
  }

  // FGMRES on K x = c for the batch's single column (x in c.x64, c in
  // c.c64); writes its iteration count and status to s_iters / s_status
  void run(double lam) {
    if (c.prm.precision != LCMG_PREC_FP64) throw ArgError("the paper's preconditioner runs in FP64 (precision = FP64)");
    pm_build(c);
    L = amg ? (int)c.am.size() : (int)c.lev.size();
    const int64_t n = c.n;
    const int m = c.prm.gmres_restart;
    c.pm_V.need((size_t)(m + 1) * n);
    c.pm_Z.need((size_t)m * n);
    c.pm_w.need(n);
    c.pm_r.need(n);
    c.pm_h.need(2 * (m + 2));
    c.pm_part.need((size_t)(m + 1) * 128);
    c.pm_y.need(m);
    setup(lam);
    // the cycle as one CUDA graph (params.graphs): it reads lambda^2, the
    // level diagonals and the coarsest inverse from device buffers that
    // setup() has filled, and runs from pm_cin into pm_cout
    cudaGraphExec_t gexec = nullptr;
    int64_t per_cycle = 0;
    if (c.prm.graphs) {
      c.pm_cin.need(n);
      c.pm_cout.need(n);
      cudaGraph_t graph = nullptr;
      const int64_t l0 = launch_counter();
      LCMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      try {
        cycle(0, c.pm_cin.p, c.pm_cout.p);
      } catch (...) {
        cudaStreamEndCapture(s, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      per_cycle = launch_counter() - l0;
      launch_counter() = l0;  // captured, not executed
      LCMG_CUDA(cudaStreamEndCapture(s, &graph));
      const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
      cudaGraphDestroy(graph);
      LCMG_CUDA(ie);
    }
    struct ExecGuard {
      cudaGraphExec_t e;
      ~ExecGuard() {
        if (e) cudaGraphExecDestroy(e);
      }
    } guard{gexec};
    auto apply_cycle = [&](const double* in, double* out) {
      if (!gexec) {
        cycle(0, in, out);
        return;
      }
      LCMG_CUDA(cudaMemcpyAsync(c.pm_cin.p, in, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      LCMG_CUDA(cudaGraphLaunch(gexec, s));
      launch_counter() += per_cycle;
      LCMG_CUDA(cudaMemcpyAsync(out, c.pm_cout.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    };
    cudaEvent_t e0, e1;
    LCMG_CUDA(cudaEventCreate(&e0));
    LCMG_CUDA(cudaEventCreate(&e1));
    LCMG_CUDA(cudaEventRecord(e0, s));
    double* x = c.x64.p;
    const double* cv = c.c64.p;
    const double cn = std::sqrt(dot(cv, cv));
    const double tol = c.prm.tol;
    const int maxit = c.prm.maxit;
    int it = 0, st = LCMG_MAXIT;
    if (cn == 0.0) {
      fill_sync(s, x, 0, sizeof(double) * n);
      st = LCMG_CONVERGED;
    }
    std::vector<double> H, g, cs, sn, hA(m + 2), hB(m + 2);
    while (cn != 0.0) {
      apply<1>(0, x, cv, c.pm_r.p, nullptr);
      const double beta = std::sqrt(dot(c.pm_r.p, c.pm_r.p));
      if (!std::isfinite(beta)) { st = LCMG_NONFINITE; break; }
      if (beta <= tol * cn) { st = LCMG_CONVERGED; break; }
      if (it >= maxit) { st = LCMG_MAXIT; break; }
      const int mm = std::min(m, maxit - it);
      klaunch(k_pm_scale, dim3(grid_for(n, 1, c.maxblk)), dim3(kBlock), 0, s, n, 1.0 / beta, (const double*)c.pm_r.p, c.pm_V.p);
      LCMG_LAUNCHED();
      H.assign((size_t)(mm + 1) * mm, 0.0);
      g.assign(mm + 1, 0.0);
      cs.assign(mm, 0.0);
      sn.assign(mm, 0.0);
      g[0] = beta;
      auto Hc = [&](int i, int j) -> double& { return H[(size_t)i * mm + j]; };
      int jd = 0;
      bool breakdown = false, nonfinite = false;
      for (int j = 0; j < mm; ++j) {
        double* vj = c.pm_V.p + (int64_t)j * n;
        double* zj = c.pm_Z.p + (int64_t)j * n;
        apply_cycle(vj, zj);
        apply<0>(0, zj, nullptr, c.pm_w.p, c.pmw[0].ppq.p);
        ++it;
        cgs_pass(j + 1, c.pm_w.p, c.pm_h.p);
        cgs_pass(j + 1, c.pm_w.p, c.pm_h.p + (m + 2));
        copy_sync(s, hA.data(), c.pm_h.p, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost);
        copy_sync(s, hB.data(), c.pm_h.p + (m + 2), sizeof(double) * (j + 1), cudaMemcpyDeviceToHost);
        for (int i = 0; i <= j; ++i) Hc(i, j) = hA[i] + hB[i];
        const double hn = std::sqrt(dot(c.pm_w.p, c.pm_w.p));
        Hc(j + 1, j) = hn;
        for (int i = 0; i <= j + 1; ++i)
          if (!std::isfinite(Hc(i, j))) nonfinite = true;
        if (nonfinite) break;
        if (hn > 0.0) {
          klaunch(k_pm_scale, dim3(grid_for(n, 1, c.maxblk)), dim3(kBlock), 0, s, n, 1.0 / hn,
                  (const double*)c.pm_w.p, c.pm_V.p + (int64_t)(j + 1) * n);
          LCMG_LAUNCHED();
        }
        for (int i = 0; i < j; ++i) {  // earlier rotations
          const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
          Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
          Hc(i, j) = t;
        }
        const double den = std::hypot(Hc(j, j), Hc(j + 1, j));
        if (den == 0.0) { breakdown = true; break; }
        cs[j] = Hc(j, j) / den;
        sn[j] = Hc(j + 1, j) / den;
        Hc(j, j) = den;
        Hc(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        jd = j + 1;
        if (std::fabs(g[j + 1]) <= tol * cn) break;
      }
      if (nonfinite) { st = LCMG_NONFINITE; break; }
      if (jd > 0) {
        std::vector<double> y(jd);
        for (int i = jd - 1; i >= 0; --i) {  // back substitution
          double t = g[i];
          for (int k2 = i + 1; k2 < jd; ++k2) t -= Hc(i, k2) * y[k2];
          y[i] = t / Hc(i, i);
        }
        copy_sync(s, c.pm_y.p, y.data(), sizeof(double) * jd, cudaMemcpyHostToDevice);
        klaunch(k_pm_combine, dim3(grid_for(n, 1, c.maxblk)), dim3(kBlock), 0, s, n, jd, (const double*)c.pm_Z.p, n,
                (const double*)c.pm_y.p, x);
        LCMG_LAUNCHED();
      }
      if (breakdown && jd == 0) { st = LCMG_BREAKDOWN; break; }
    }
    LCMG_CUDA(cudaEventRecord(e1, s));
    LCMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.stats.iterate_ms += ms;
    c.stats.batch_iterations += it;
    copy_sync(s, c.s_iters.p, &it, sizeof(int), cudaMemcpyHostToDevice);
    copy_sync(s, c.s_status.p, &st, sizeof(int), cudaMemcpyHostToDevice);
  }
};

// Solve the columns cols (each = (lambda index li, rhs index ri)) as one
// batch.  x0p: planar initial guesses per column (device, may be null) ;
// outputs planar per column.
struct ColSpec {
  double lam;
  int rhs;
};

static void solve_columns(lcmg_ctx& c, const std::vector<ColSpec>& cols, int nrhs,
                          const std::vector<const double*>& x0, const std::vector<double*>& xout,
                          double* rho, double* eta, int* iters, int* status) {
  const int B = (int)cols.size();
  if (c.prm.precond == 1 && B > 1) {  // the paper's method: one column at a time
    for (int j = 0; j < B; ++j)
      solve_columns(c, {cols[j]}, nrhs, {x0[j]}, {xout[j]}, rho ? rho + j : nullptr, eta ? eta + j : nullptr,
                    iters ? iters + j : nullptr, status ? status + j : nullptr);
    return;
  }
  ensure_work(c, B);
  cudaStream_t s = c.stream;
  // column pointer tables and the column -> right-hand-side map
  std::vector<const double*> hptr(2 * B);
  std::vector<int> hmap(B);
  for (int j = 0; j < B; ++j) {
    hptr[j] = x0[j];
    hptr[B + j] = xout[j];
    hmap[j] = cols[j].rhs;
  }
  const double** dptr = static_cast<const double**>(static_cast<void*>(c.colptr.need(2 * B)));
  int* dmap = c.colmap.need(B);
  LCMG_CUDA(cudaMemcpyAsync(dptr, hptr.data(), sizeof(double*) * 2 * B, cudaMemcpyHostToDevice, s));
  LCMG_CUDA(cudaMemcpyAsync(dmap, hmap.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  const int gn = grid_for(c.n, B, c.maxblk);
  klaunch(k_gather_cols, dim3(gn), dim3(kBlock), 0, s, c.n, B, dptr, c.x64.p);
  LCMG_LAUNCHED();
  klaunch(k_gather_map, dim3(gn), dim3(kBlock), 0, s, c.n, B, nrhs, dmap, c.cvec.p, c.c64.p);
  LCMG_LAUNCHED();
  LCMG_CUDA(cudaStreamSynchronize(s));  // host tables must outlive the copies
  std::vector<double> lam(B);
  for (int j = 0; j < B; ++j) lam[j] = cols[j].lam;
  if (c.prm.precond == 1) {
    PaperMG(c).run(lam[0]);
  } else if (c.prm.precision == LCMG_PREC_FP64) {
    Batch<double> b(c, B);
    b.run(lam);
  } else {
    Batch<float> b(c, B);
    b.run(lam);
  }
  // outputs: x (the pointer table is unchanged since the gather)
  klaunch(k_scatter_cols, dim3(gn), dim3(kBlock), 0, s, c.n, B, c.x64.p, c.colptr.p + B);
  LCMG_LAUNCHED();
  // rho = ||A x - b|| per column: b of each column's right-hand side
  double* bcol = c.y64.p;  // [m][B]
  klaunch(k_gather_map, dim3(grid_for(c.m, B, c.maxblk)), dim3(kBlock), 0, s, c.m, B, nrhs, dmap, c.bvec.p, bcol);
  LCMG_LAUNCHED();
  int nb;
  if (c.fwd == 1) {
    SpmmArgs a = csr_args(c, false, B);
    a.nrhs = B;
    FineOp<double> f = view<double>(c, 0).fine_op();
    if (c.vdtype == 1)
      nb = launch_spmm<double, double, double, 2>(a, c.v64.p, c.x64.p, (double*)nullptr, f, nullptr, nullptr,
                                                  nullptr, bcol, c.part_x.p, c.maxblk, s);
    else
      nb = launch_spmm<float, double, double, 2>(a, c.v32.p, c.x64.p, (double*)nullptr, f, nullptr, nullptr,
                                                 nullptr, bcol, c.part_x.p, c.maxblk, s);
  } else if (c.sep) {
    // A x = (A_h (x) A_v) x along i, then j with the partials of (A x - b)^2
    double* tmp = c.sep_tmp.need((size_t)c.n * B);
    FineOp<double> f = view<double>(c, 0).fine_op();
    launch_band<double, double, 0, BAND_STORE>(c.nv, c.nh, B, make_band<double>(c.sp_va, nullptr), c.x64.p, tmp, f,
                                               nullptr, nullptr, nullptr, nullptr, nullptr, c.maxblk, s);
    nb = launch_band<double, double, 1, BAND_RESID2>(c.nv, c.nh, B, make_band<double>(c.sp_ha, nullptr), tmp,
                                                     (double*)nullptr, f, nullptr, nullptr, nullptr, bcol, c.part_x.p,
                                                     c.maxblk, s);
  } else {
    PsfArgs pa{};
    pa.nv = c.nv; pa.nh = c.nh; pa.rv = c.rv; pa.rh = c.rh; pa.psf = c.psf64.p;
    nb = grid_for(c.n, B, c.maxblk);
    klaunch(k_psf_forward<double, 2>, dim3(nb), dim3(kBlock), 0, s, pa, c.psf64.p, B, c.x64.p, nullptr, bcol, 1, B, c.part_x.p);
    LCMG_LAUNCHED();
  }
  klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, s, B, nb, c.part_x.p, c.s_out.p);
  LCMG_LAUNCHED();
  std::vector<double> hr(B), he(B);
  LCMG_CUDA(cudaMemcpyAsync(hr.data(), c.s_out.p, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  const int g = grid_for(c.n, B, c.maxblk);
  klaunch(k_seminorm, dim3(g), dim3(kBlock), 0, s, c.nv, c.nh, B, c.ws.p, c.we.p, c.x64.p, c.part_x.p);
  LCMG_LAUNCHED();
  klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, s, B, g, c.part_x.p, c.s_out.p);
  LCMG_LAUNCHED();
  LCMG_CUDA(cudaMemcpyAsync(he.data(), c.s_out.p, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  std::vector<int> hi(B), hs(B);
  LCMG_CUDA(cudaMemcpyAsync(hi.data(), c.s_iters.p, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  LCMG_CUDA(cudaMemcpyAsync(hs.data(), c.s_status.p, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  LCMG_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < B; ++j) {
    if (rho) rho[j] = std::sqrt(hr[j]);
    if (eta) eta[j] = std::sqrt(he[j]);
    if (iters) iters[j] = hi[j];
    if (status) status[j] = hs[j] == ST_RUNNING ? ST_MAXIT : hs[j];
    c.stats.column_iterations += hi[j];
  }
}

static void require_ready(lcmg_ctx& c) {
  if (c.nv == 0) throw ArgError("set_grid has not been called");
  if (c.fwd == 0) throw ArgError("forward operator not set");
  ensure_hierarchy(c);
}

static void check_lambdas(int nl, const double* lam) {
  if (nl < 1 || !lam) throw ArgError("empty lambda list");
  for (int i = 0; i < nl; ++i) {
    if (!(lam[i] > 0.0) || !std::isfinite(lam[i])) throw ArgError("lambdas must be positive and finite");
    if (i > 0 && !(lam[i] > lam[i - 1])) throw ArgError("lambdas must be strictly increasing");
  }
}

// Solve for all (lambda, rhs) pairs; b_dev interleaved already in c.bvec and
// c.cvec computed.  x0/x: device planar [nrhs][nl][n].
static void solve_all(lcmg_ctx& c, int nl, const double* lam, int nrhs, const double* x0, double* x,
                      double* rho, double* eta, int* iters, int* status) {
  const int64_t n = c.n;
  if (c.prm.mode == LCMG_MODE_BATCHED) {
    const int total = nl * nrhs;
    for (int start = 0; start < total; start += kMaxB) {
      const int cnt = std::min(kMaxB, total - start);
      std::vector<ColSpec> cols(cnt);
      std::vector<const double*> x0s(cnt);
      std::vector<double*> xs(cnt);
      for (int j = 0; j < cnt; ++j) {
        const int idx = start + j;  // idx = r * nl + li
        cols[j].rhs = idx / nl;
        cols[j].lam = lam[idx % nl];
        x0s[j] = x0 ? x0 + (int64_t)idx * n : nullptr;
        xs[j] = x + (int64_t)idx * n;
      }
      solve_columns(c, cols, nrhs, x0s, xs, rho ? rho + start : nullptr, eta ? eta + start : nullptr,
                    iters ? iters + start : nullptr, status ? status + start : nullptr);
    }
    return;
  }
  // sequential: largest lambda first, each right-hand side warm-started
  // from its own solution at the previous lambda (Sec. 3.3), the first from
  // x0 (if given).  The chains of the right-hand sides advance together: at
  // each lambda one batch holds every right-hand side's system (they share
  // lambda, so the operator, the hierarchy and its coefficients are read
  // once for all of them); per column the iteration is the chain's own.
  for (int r0 = 0; r0 < nrhs; r0 += kMaxB) {
    const int cnt = std::min(kMaxB, nrhs - r0);
    std::vector<const double*> prev(cnt, nullptr);
    for (int li = nl - 1; li >= 0; --li) {
      std::vector<ColSpec> cols(cnt);
      std::vector<const double*> x0s(cnt);
      std::vector<double*> xs(cnt);
      std::vector<double> rh(cnt), eh(cnt);
      std::vector<int> ih(cnt), sh(cnt);
      for (int j = 0; j < cnt; ++j) {
        const int64_t idx = (int64_t)(r0 + j) * nl + li;
        cols[j] = ColSpec{lam[li], r0 + j};
        x0s[j] = prev[j] ? prev[j] : (x0 ? x0 + idx * n : nullptr);
        xs[j] = x + idx * n;
      }
      solve_columns(c, cols, nrhs, x0s, xs, rh.data(), eh.data(), ih.data(), sh.data());
      for (int j = 0; j < cnt; ++j) {
        const int64_t idx = (int64_t)(r0 + j) * nl + li;
        if (rho) rho[idx] = rh[j];
        if (eta) eta[idx] = eh[j];
        if (iters) iters[idx] = ih[j];
        if (status) status[idx] = sh[j];
        prev[j] = xs[j];
      }
    }
  }
}

static void upload_b(lcmg_ctx& c, int nrhs, const double* b, bool dev) {
  // b planar [nrhs][m] -> interleaved [m][nrhs]
  double* bi = c.bvec.need((size_t)c.m * nrhs);
  const double* src = b;
  if (!dev) {
    double* tmp = c.stage_b.need((size_t)c.m * nrhs);
    LCMG_CUDA(cudaMemcpyAsync(tmp, b, sizeof(double) * c.m * nrhs, cudaMemcpyHostToDevice, c.stream));
    src = tmp;
  }
  klaunch(k_planar_to_inter, dim3(grid_for(c.m, nrhs, c.maxblk)), dim3(kBlock), 0, c.stream, c.m, nrhs, src, bi);
  LCMG_LAUNCHED();
  compute_rhs(c, nrhs);
  LCMG_CUDA(cudaStreamSynchronize(c.stream));
}

// ---------------------------------------------------------------------------
// L-curve corner (host; reading of Sec. 1 stated in lcmg.h)
// ---------------------------------------------------------------------------
static int corner_host(int k, const double* rho, const double* eta) {
  std::vector<double> u(k), v(k), kap(k, -INFINITY);
  for (int i = 0; i < k; ++i) { u[i] = std::log10(rho[i]); v[i] = std::log10(eta[i]); }
  for (int i = 1; i + 1 < k; ++i) {
    const double ax = u[i] - u[i - 1], ay = v[i] - v[i - 1];
    const double bx = u[i + 1] - u[i], by = v[i + 1] - v[i];
    const double cx = u[i + 1] - u[i - 1], cy = v[i + 1] - v[i - 1];
    const double cross = ax * by - ay * bx;
    const double den = std::hypot(ax, ay) * std::hypot(bx, by) * std::hypot(cx, cy);
    kap[i] = den > 0 ? 2.0 * cross / den : 0.0;
  }
  bool anypos = false;
  for (int i = 1; i + 1 < k; ++i) anypos |= kap[i] > 0;
  int best = -1;
  for (int i = 1; i + 1 < k; ++i) {
    if (anypos && !(kap[i] > 0)) continue;
    if (best < 0 || kap[i] > kap[best] + 1e-12 * std::fabs(kap[best])) best = i;
  }
  return best;
}

static void window(int m, int i_prev, int* lo, int* hi) {
  if (i_prev <= 0) { *lo = 1; *hi = m; return; }
  *lo = std::max(std::min(i_prev - 2, m - 9), 1);
  *hi = std::min(std::max(i_prev + 7, 10), m);
}

static void update_weights_dev(lcmg_ctx& c, const double* xs, double q, double dmin) {
  if (!(q > 0.0) || !(dmin > 0.0 && dmin <= 1.0)) throw ArgError("q must be > 0 and d_min in (0, 1]");
  const int g = (int)std::min<int64_t>((c.ne + kBlock - 1) / kBlock, c.maxblk);
  double* absv = c.absv.need(c.ne);
  double* bmax = c.bmax.need(g);
  klaunch(k_weighted_grad, dim3(g), dim3(kBlock), 0, c.stream, c.nv, c.nh, c.d.p, xs, absv, bmax);
  LCMG_LAUNCHED();
  klaunch(k_weight_apply, dim3(g), dim3(kBlock), 0, c.stream, c.ne, g, bmax, absv, q, dmin, c.d.p);
  LCMG_LAUNCHED();
  refresh_fine(c);
}

// Statistics of one top-level call: reset at entry, launches counted at exit.
struct StatsScope {
  lcmg_ctx& c;
  int64_t l0;
  explicit StatsScope(lcmg_ctx& c_) : c(c_), l0(launch_counter()) { c.stats = lcmg_stats{}; }
  ~StatsScope() { c.stats.kernel_launches = launch_counter() - l0; }
};

// ||L x||_2 of one device vector (unweighted gradient)
static double grad_norm(lcmg_ctx& c, const double* x) {
  double* ones = c.ones.need(c.n);
  if (!c.ones_ok) {
    std::vector<double> h(c.n, 1.0);
    copy_sync(c.stream, ones, h.data(), sizeof(double) * c.n, cudaMemcpyHostToDevice);
    c.ones_ok = true;
  }
  const int g = grid_for(c.n, 1, c.maxblk);
  klaunch(k_seminorm, dim3(g), dim3(kBlock), 0, c.stream, c.nv, c.nh, 1, ones, ones, x, c.part_x.p);
  LCMG_LAUNCHED();
  klaunch(k_sum_parts, dim3(1), dim3(kScalarThreads), 0, c.stream, 1, g, c.part_x.p, c.s_out.p);
  LCMG_LAUNCHED();
  double v = 0.0;
  copy_sync(c.stream, &v, c.s_out.p, sizeof(double), cudaMemcpyDeviceToHost);
  return std::sqrt(v);
}

static void lcurve_run_impl(lcmg_ctx& c, int m, const double* lam, int max_outer, double* x_out_dev,
                            int* hist, int* n_outer, int64_t* n_solves, int64_t* n_conv) {
  check_lambdas(m, lam);
  if (max_outer < 1) throw ArgError("max_outer must be >= 1");
  const int64_t n = c.n;
  DevBuf<double>& xres = c.run_xres;
  DevBuf<double>& xstar = c.run_xstar;
  DevBuf<double>& xwin = c.run_xwin;
  xres.need((size_t)m * n);
  xstar.need(n);
  LCMG_CUDA(cudaMemsetAsync(xstar.p, 0, sizeof(double) * n, c.stream));
  std::vector<int> solved(m, 0);
  std::vector<int> h;
  std::vector<double> lx;  // ||L x*||_2 per outer iteration (stop_rule 1)
  int64_t ns = 0, nconv = 0;
  int ell = 0;
  for (ell = 1; ell <= max_outer; ++ell) {
    int lo, hi;
    window(m, h.empty() ? 0 : h.back(), &lo, &hi);
    const int k = hi - lo + 1;
    ensure_hierarchy(c);
    xwin.need((size_t)k * n);
    std::vector<double> rho(k), eta(k);
    std::vector<int> its(k), st(k);
    if (c.prm.mode == LCMG_MODE_BATCHED) {
      // each lambda starts from its own previous solution, else from x*
      std::vector<ColSpec> cols(k);
      std::vector<const double*> x0s(k);
      std::vector<double*> xs(k);
      for (int j = 0; j < k; ++j) {
        const int i = lo + j;  // 1-based
        cols[j] = ColSpec{lam[i - 1], 0};
        x0s[j] = solved[i - 1] ? xres.p + (int64_t)(i - 1) * n : xstar.p;
        xs[j] = xwin.p + (int64_t)j * n;
      }
      solve_columns(c, cols, 1, x0s, xs, rho.data(), eta.data(), its.data(), st.data());
    } else {
      // largest first, chained; the first from x*
      const double* prev = xstar.p;
      for (int j = k - 1; j >= 0; --j) {
        std::vector<ColSpec> cols{{lam[lo + j - 1], 0}};
        std::vector<const double*> x0s{prev};
        std::vector<double*> xs{xwin.p + (int64_t)j * n};
        solve_columns(c, cols, 1, x0s, xs, &rho[j], &eta[j], &its[j], &st[j]);
        prev = xwin.p + (int64_t)j * n;
      }
    }
    for (int j = 0; j < k; ++j) {
      LCMG_CUDA(cudaMemcpyAsync(xres.p + (int64_t)(lo + j - 1) * n, xwin.p + (int64_t)j * n, sizeof(double) * n,
                                cudaMemcpyDeviceToDevice, c.stream));
      solved[lo + j - 1] = 1;
      ns += 1;
      nconv += st[j] == 0;
    }
    const int sel = lo + corner_host(k, rho.data(), eta.data());
    h.push_back(sel);
    LCMG_CUDA(cudaMemcpyAsync(xstar.p, xwin.p + (int64_t)(sel - lo) * n, sizeof(double) * n,
                              cudaMemcpyDeviceToDevice, c.stream));
    const int L = (int)h.size();
    if (c.prm.stop_rule == 1) {
      lx.push_back(grad_norm(c, xstar.p));
      if (L >= 2 && lx[L - 1] < lx[L - 2]) break;
    } else if (L >= 3 && h[L - 1] == h[L - 2] && h[L - 2] == h[L - 3]) {
      break;
    }
    if (ell == max_outer) break;
    update_weights_dev(c, xstar.p, c.prm.q, c.prm.d_min);
  }
  LCMG_CUDA(cudaMemcpyAsync(x_out_dev, xstar.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.stream));
  LCMG_CUDA(cudaStreamSynchronize(c.stream));
  for (size_t i = 0; i < h.size(); ++i) hist[i] = h[i];
  *n_outer = (int)h.size();
  if (n_solves) *n_solves = ns;
  if (n_conv) *n_conv = nconv;
}

}  // namespace lcmg

// ===========================================================================
// C ABI
// ===========================================================================
#define API_BEGIN try {
#define API_END                                                    \
  }                                                                \
  catch (const lcmg::ArgError& e) {                                \
    lcmg::set_err(e.what());                                       \
    return LCMG_ERR_INVALID_ARG;                                   \
  }                                                                \
  catch (const lcmg::MemError& e) {                                \
    lcmg::set_err(e.what());                                       \
    return LCMG_ERR_NOMEM;                                         \
  }                                                                \
  catch (const lcmg::CudaError& e) {                               \
    lcmg::set_err(e.what());                                       \
    return LCMG_ERR_CUDA;                                          \
  }                                                                \
  catch (const std::exception& e) {                                \
    lcmg::set_err(e.what());                                       \
    return LCMG_ERR_STATE;                                         \
  }                                                                \
  lcmg::g_err.clear();                                             \
  return LCMG_OK;

#define NEED_CTX() \
  if (!ctx) throw lcmg::ArgError("null context")

extern "C" {

void lcmg_default_params(lcmg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->levels = 0;
  p->coarse_max = 16;
  p->nu = 1;
  p->smoother = LCMG_SMOOTH_L1_JACOBI;
  p->omega = 2.0 / 3.0;
  p->q = 2.0;
  p->d_min = 1e-3;
  p->tol = 1e-6;
  p->maxit = 10000;
  p->precision = LCMG_PREC_FP64;
  p->mode = LCMG_MODE_SEQUENTIAL;
  p->check_every = 16;
  p->graphs = 1;
  p->timing = 0;
  p->vfuse = 1;
  p->keep_direction = 0;
  p->autotune = 0;
  p->spmv_variant = 0;
  p->stop_rule = 0;
  p->precond = 0;
  p->gmres_restart = 200;
  p->coarsening = 0;
  p->amg_coarse_max = 256;
  p->compact_cols = 1;
  p->alpha_fuse = 1;
  p->beta_fuse = 1;
  p->spmv_variant_at = 0;
  p->max_blocks = 0;
  p->smoother_fp16 = 1;
}

const char* lcmg_last_error(void) { return lcmg::g_err.c_str(); }
const char* lcmg_version(void) { return "lcmg 0.1 (sm_103a)"; }

int lcmg_create(lcmg_ctx** out, int device, void* stream, const lcmg_params* p) {
  API_BEGIN
  if (!out) throw lcmg::ArgError("null output pointer");
  *out = nullptr;
  int ndev = 0;
  LCMG_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) throw lcmg::ArgError("invalid device");
  LCMG_CUDA(cudaSetDevice(device));
  lcmg_params prm;
  lcmg_default_params(&prm);
  if (p) prm = *p;
  lcmg::check_params(prm);
  auto* c = new lcmg_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (!c->stream) {
    // a stream of our own, non-blocking: no implicit synchronisation with
    // the legacy stream, so other threads' work never joins our captures
    LCMG_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  c->prm = prm;
  cudaDeviceProp prop;
  LCMG_CUDA(cudaGetDeviceProperties(&prop, device));
  c->sms = prop.multiProcessorCount;
  c->maxblk = std::min(lcmg::kMaxBlocks, c->sms * 8);
  if (prm.max_blocks > 0) c->maxblk = std::min(c->maxblk, prm.max_blocks);
  *out = c;
  API_END
}

int lcmg_destroy(lcmg_ctx* ctx) {
  API_BEGIN
  if (!ctx) return LCMG_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
  for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  API_END
}

int lcmg_set_params(lcmg_ctx* ctx, const lcmg_params* p) {
  API_BEGIN
  NEED_CTX();
  if (!p) throw lcmg::ArgError("null params");
  lcmg::check_params(*p);
  const bool lev_change = p->levels != ctx->prm.levels || p->coarse_max != ctx->prm.coarse_max ||
                          p->coarsening != ctx->prm.coarsening;
  const bool amg_change = lev_change || p->amg_coarse_max != ctx->prm.amg_coarse_max;
  ctx->prm = *p;
  ctx->maxblk = std::min(lcmg::kMaxBlocks, ctx->sms * 8);
  if (p->max_blocks > 0) ctx->maxblk = std::min(ctx->maxblk, p->max_blocks);
  if (lev_change) ctx->hier_ok = false;
  if (amg_change) {
    ctx->am_ok = false;
    ctx->pm_levels = 0;
  }
  API_END
}

int lcmg_set_grid(lcmg_ctx* ctx, int32_t n_v, int32_t n_h) {
  API_BEGIN
  NEED_CTX();
  if (n_v < 2 || n_h < 2) throw lcmg::ArgError("grid sides must be >= 2");
  LCMG_CUDA(cudaSetDevice(ctx->device));
  ctx->nv = n_v;
  ctx->nh = n_h;
  ctx->n = (int64_t)n_v * n_h;
  ctx->ne = (int64_t)n_h * (n_v - 1) + (int64_t)(n_h - 1) * n_v;
  ctx->fwd = 0;
  ctx->c16_ok = false;
  ctx->tuned.clear();
  ctx->ones_ok = false;
  ctx->pm_levels = 0;
  ctx->am_ok = false;
  std::vector<double> ones(ctx->ne, 1.0);
  lcmg::copy_sync(ctx->stream, ctx->d.need(ctx->ne), ones.data(), sizeof(double) * ctx->ne, cudaMemcpyHostToDevice);
  lcmg::refresh_fine(*ctx);
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  API_END
}

int lcmg_set_forward_csr(lcmg_ctx* ctx, int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const void* val, int32_t val_dtype) {
  API_BEGIN
  NEED_CTX();
  if (ctx->nv == 0) throw lcmg::ArgError("set_grid has not been called");
  if (n != ctx->n) throw lcmg::ArgError("n must equal n_v * n_h");
  if (m < 1 || !row_ptr || !col || !val) throw lcmg::ArgError("bad CSR arguments");
  if (val_dtype != 0 && val_dtype != 1) throw lcmg::ArgError("val_dtype must be 0 (FP32) or 1 (FP64)");
  if (row_ptr[0] != 0) throw lcmg::ArgError("row_ptr[0] must be 0");
  for (int64_t i = 0; i < m; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) throw lcmg::ArgError("row_ptr must be non-decreasing");
  const int64_t nnz = row_ptr[m];
  std::vector<int64_t> cnt(n + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) {
    if (col[k] < 0 || col[k] >= n) throw lcmg::ArgError("column index out of range");
    cnt[col[k] + 1]++;
  }
  LCMG_CUDA(cudaSetDevice(ctx->device));
  // transposed CSR by a stable counting sort on the column index
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int64_t> rpT(cnt.begin(), cnt.end());
  std::vector<int32_t> ciT(nnz);
  std::vector<double> vT(nnz);
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  const float* vf = static_cast<const float*>(val);
  const double* vd = static_cast<const double*>(val);
  for (int64_t r = 0; r < m; ++r)
    for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
      const int64_t dst = pos[col[k]]++;
      ciT[dst] = (int32_t)r;
      vT[dst] = val_dtype == 0 ? (double)vf[k] : vd[k];
    }
  ctx->m = m;
  ctx->nnz = nnz;
  ctx->vdtype = val_dtype;
  cudaStream_t s = ctx->stream;
  // CSR arrays padded by kCsrPad elements (vector loads may run past the last row)
  lcmg::copy_sync(ctx->stream, ctx->rp.need(m + 1 + lcmg::kCsrPad), row_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice);
  lcmg::copy_sync(ctx->stream, ctx->ci.need(nnz + lcmg::kCsrPad), col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice);
  lcmg::copy_sync(ctx->stream, ctx->rpT.need(n + 1 + lcmg::kCsrPad), rpT.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
  lcmg::copy_sync(ctx->stream, ctx->ciT.need(nnz + lcmg::kCsrPad), ciT.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice);
  std::vector<float> tmpf(nnz);
  if (val_dtype == 0) {
    lcmg::copy_sync(ctx->stream, ctx->v32.need(nnz + lcmg::kCsrPad), vf, sizeof(float) * nnz, cudaMemcpyHostToDevice);
  } else {
    lcmg::copy_sync(ctx->stream, ctx->v64.need(nnz + lcmg::kCsrPad), vd, sizeof(double) * nnz, cudaMemcpyHostToDevice);
    lcmg::copy_sync(ctx->stream, ctx->vT64.need(nnz + lcmg::kCsrPad), vT.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice);
    for (int64_t k = 0; k < nnz; ++k) tmpf[k] = (float)vd[k];
    lcmg::copy_sync(ctx->stream, ctx->v32.need(nnz + lcmg::kCsrPad), tmpf.data(), sizeof(float) * nnz, cudaMemcpyHostToDevice);
  }
  for (int64_t k = 0; k < nnz; ++k) tmpf[k] = (float)vT[k];
  lcmg::copy_sync(ctx->stream, ctx->vT32.need(nnz + lcmg::kCsrPad), tmpf.data(), sizeof(float) * nnz, cudaMemcpyHostToDevice);
  // 16-bit column offsets when every row of A and of A^T spans fewer than
  // 65,536 columns (base = the row's smallest column)
  {
    auto compact = [&](int64_t rows, const int64_t* rp, const int32_t* ci, std::vector<int32_t>& base,
                       std::vector<uint16_t>& off) {
      base.assign(rows, 0);
      off.assign(nnz, 0);
      for (int64_t r = 0; r < rows; ++r) {
        if (rp[r + 1] == rp[r]) continue;
        int32_t mn = ci[rp[r]], mx = mn;
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
          mn = std::min(mn, ci[k]);
          mx = std::max(mx, ci[k]);
        }
        if ((int64_t)mx - mn > 65535) return false;
        base[r] = mn;
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k) off[k] = (uint16_t)(ci[k] - mn);
      }
      return true;
    };
    std::vector<int32_t> b1, b2;
    std::vector<uint16_t> o1, o2;
    ctx->c16_ok = compact(m, row_ptr, col, b1, o1) && compact(n, rpT.data(), ciT.data(), b2, o2);
    if (ctx->c16_ok) {
      lcmg::copy_sync(s, ctx->c16.need(nnz + lcmg::kCsrPad), o1.data(), sizeof(uint16_t) * nnz, cudaMemcpyHostToDevice);
      lcmg::copy_sync(s, ctx->c16T.need(nnz + lcmg::kCsrPad), o2.data(), sizeof(uint16_t) * nnz, cudaMemcpyHostToDevice);
      lcmg::copy_sync(s, ctx->rbase.need(m), b1.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice);
      lcmg::copy_sync(s, ctx->rbaseT.need(n), b2.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
    } else {
      ctx->c16.release(); ctx->c16T.release(); ctx->rbase.release(); ctx->rbaseT.release();
    }
  }
  // zero padding after the last nonzero (read by the 16-byte vector loads)
  lcmg::fill_sync(ctx->stream, ctx->ci.p + nnz, 0, sizeof(int32_t) * lcmg::kCsrPad);
  lcmg::fill_sync(ctx->stream, ctx->ciT.p + nnz, 0, sizeof(int32_t) * lcmg::kCsrPad);
  lcmg::fill_sync(ctx->stream, ctx->v32.p + nnz, 0, sizeof(float) * lcmg::kCsrPad);
  lcmg::fill_sync(ctx->stream, ctx->vT32.p + nnz, 0, sizeof(float) * lcmg::kCsrPad);
  if (val_dtype == 1) {
    lcmg::fill_sync(ctx->stream, ctx->v64.p + nnz, 0, sizeof(double) * lcmg::kCsrPad);
    lcmg::fill_sync(ctx->stream, ctx->vT64.p + nnz, 0, sizeof(double) * lcmg::kCsrPad);
  }
  // diag(A^T A): sums of squares along the rows of A^T
  const int g = (int)std::min<int64_t>((n * 32 + lcmg::kBlock - 1) / lcmg::kBlock, ctx->maxblk);
  if (val_dtype == 1)
    klaunch(lcmg::k_diag_ata<double>, dim3(g), dim3(lcmg::kBlock), 0, s, n, ctx->rpT.p, ctx->vT64.p, ctx->diag.need(n));
  else
    klaunch(lcmg::k_diag_ata<float>, dim3(g), dim3(lcmg::kBlock), 0, s, n, ctx->rpT.p, ctx->vT32.p, ctx->diag.need(n));
  LCMG_LAUNCHED();
  klaunch(lcmg::k_convert<double, float>, dim3(g), dim3(lcmg::kBlock), 0, s, n, ctx->diag.p, ctx->diag32.need(n));
  LCMG_LAUNCHED();
  LCMG_CUDA(cudaStreamSynchronize(s));
  ctx->fwd = 1;
  ctx->hier_ok = false;
  ctx->tuned.clear();
  ctx->pm_levels = 0;
  ctx->am_ok = false;
  API_END
}

namespace lcmg {
// psf = fv fh^T to rounding?  fv = the row sums, fh = the column sums over
// their total (exact for an outer product); accepted when every entry
// matches the product within 1e-14 of the largest entry
static bool rank_one(int kh, int kw, const double* psf, std::vector<double>& fv, std::vector<double>& fh) {
  fv.assign(kh, 0.0);
  fh.assign(kw, 0.0);
  double tot = 0.0, amax = 0.0;
  for (int u = 0; u < kh; ++u)
    for (int v = 0; v < kw; ++v) {
      fv[u] += psf[u * kw + v];
      fh[v] += psf[u * kw + v];
      tot += psf[u * kw + v];
      amax = std::max(amax, std::fabs(psf[u * kw + v]));
    }
  if (!(tot != 0.0) || amax == 0.0) return false;
  for (double& x : fh) x /= tot;
  for (int u = 0; u < kh; ++u)
    for (int v = 0; v < kw; ++v)
      if (std::fabs(psf[u * kw + v] - fv[u] * fh[v]) > 1e-14 * amax) return false;
  return true;
}

// The blur A = A_h (x) A_v of the 1-D correlations fv (along i) and fh
// (along j), Sec. 4: banded passes of A^T A, A and A^T, their boundary
// correction rows on the device, diag(A^T A) = T_v[i][i] T_h[j][j]
static void set_separable(lcmg_ctx* c, const std::vector<double>& fv, const std::vector<double>& fh) {
  c->sp_vt = sep_pass_ata(fv, c->nv);
  c->sp_ht = sep_pass_ata(fh, c->nh);
  c->sp_va = sep_pass_corr(fv, false);
  c->sp_ha = sep_pass_corr(fh, false);
  c->sp_vat = sep_pass_corr(fv, true);
  c->sp_hat = sep_pass_corr(fh, true);
  auto up = [&](const std::vector<double>& d, DevBuf<double>& b64, DevBuf<float>& b32) {
    std::vector<float> f32(d.begin(), d.end());
    copy_sync(c->stream, b64.need(d.size()), d.data(), sizeof(double) * d.size(), cudaMemcpyHostToDevice);
    copy_sync(c->stream, b32.need(d.size()), f32.data(), sizeof(float) * d.size(), cudaMemcpyHostToDevice);
  };
  up(c->sp_vt.d, c->sep_dv64, c->sep_dv32);
  up(c->sp_ht.d, c->sep_dh64, c->sep_dh32);
  const std::vector<double> dv = sep_diag(c->sp_vt, c->nv), dh = sep_diag(c->sp_ht, c->nh);
  DevBuf<double> ddv, ddh;
  copy_sync(c->stream, ddv.need(dv.size()), dv.data(), sizeof(double) * dv.size(), cudaMemcpyHostToDevice);
  copy_sync(c->stream, ddh.need(dh.size()), dh.data(), sizeof(double) * dh.size(), cudaMemcpyHostToDevice);
  launch_sep_diag(c->nv, c->nh, ddv.p, ddh.p, c->diag.need(c->n), c->maxblk, c->stream);
  LCMG_CUDA(cudaStreamSynchronize(c->stream));
  prepare_band();
  c->sep = true;
}

// common part of the stencil setters: store the 2-D PSF, pick the form
static void set_stencil(lcmg_ctx* ctx, int32_t kh, int32_t kw, const double* psf, const std::vector<double>* fv,
                        const std::vector<double>* fh) {
  if (ctx->nv == 0) throw ArgError("set_grid has not been called");
  if (kh > 2 * ctx->nv + 1 || kw > 2 * ctx->nh + 1) throw ArgError("PSF larger than the image");
  for (int i = 0; i < kh * kw; ++i)
    if (!std::isfinite(psf[i])) throw ArgError("PSF values must be finite");
  LCMG_CUDA(cudaSetDevice(ctx->device));
  ctx->rv = kh / 2;
  ctx->rh = kw / 2;
  ctx->m = ctx->n;
  ctx->sep = false;
  copy_sync(ctx->stream, ctx->psf64.need(kh * kw), psf, sizeof(double) * kh * kw, cudaMemcpyHostToDevice);
  std::vector<float> pf(psf, psf + kh * kw);
  copy_sync(ctx->stream, ctx->psf32.need(kh * kw), pf.data(), sizeof(float) * kh * kw, cudaMemcpyHostToDevice);
  std::vector<double> av, ah;
  const bool fits = 2 * ctx->rv <= kBandMaxH && 2 * ctx->rh <= kBandMaxH;
  if (fits && fv) {
    set_separable(ctx, *fv, *fh);
  } else if (fits && rank_one(kh, kw, psf, av, ah)) {
    set_separable(ctx, av, ah);
  } else {
    PsfArgs pa{};
    pa.nv = ctx->nv; pa.nh = ctx->nh; pa.rv = ctx->rv; pa.rh = ctx->rh; pa.psf = ctx->psf64.p;
    const int g = (int)std::min<int64_t>((ctx->n + kBlock - 1) / kBlock, ctx->maxblk);
    klaunch(k_psf_diag, dim3(g), dim3(kBlock), 0, ctx->stream, pa, ctx->diag.need(ctx->n));
    LCMG_LAUNCHED();
  }
  const int g = (int)std::min<int64_t>((ctx->n + kBlock - 1) / kBlock, ctx->maxblk);
  klaunch(k_convert<double, float>, dim3(g), dim3(kBlock), 0, ctx->stream, ctx->n, ctx->diag.p,
          ctx->diag32.need(ctx->n));
  LCMG_LAUNCHED();
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->fwd = 2;
  ctx->c16_ok = false;
  ctx->tuned.clear();
  ctx->pm_levels = 0;
  ctx->am_ok = false;
  ctx->hier_ok = false;
}
}  // namespace lcmg

int lcmg_set_forward_stencil(lcmg_ctx* ctx, int32_t kh, int32_t kw, const double* psf) {
  API_BEGIN
  NEED_CTX();
  if (kh < 1 || kw < 1 || kh % 2 == 0 || kw % 2 == 0 || !psf) throw lcmg::ArgError("PSF sides must be odd");
  lcmg::set_stencil(ctx, kh, kw, psf, nullptr, nullptr);
  API_END
}

int lcmg_set_forward_separable(lcmg_ctx* ctx, int32_t kh, const double* fv, int32_t kw, const double* fh) {
  API_BEGIN
  NEED_CTX();
  if (kh < 1 || kw < 1 || kh % 2 == 0 || kw % 2 == 0 || !fv || !fh)
    throw lcmg::ArgError("filter lengths must be odd");
  std::vector<double> a(fv, fv + kh), b(fh, fh + kw), psf((size_t)kh * kw);
  for (int u = 0; u < kh; ++u)
    for (int v = 0; v < kw; ++v) psf[(size_t)u * kw + v] = a[u] * b[v];
  lcmg::set_stencil(ctx, kh, kw, psf.data(), &a, &b);
  API_END
}

int lcmg_forward_form(lcmg_ctx* ctx, int32_t* form) {
  API_BEGIN
  NEED_CTX();
  if (!form) throw lcmg::ArgError("null output pointer");
  *form = ctx->fwd == 2 ? (ctx->sep ? 3 : 2) : ctx->fwd;
  API_END
}

static void set_weights_common(lcmg_ctx* ctx, const double* d, int64_t n_edges, bool dev) {
  if (ctx->nv == 0) throw lcmg::ArgError("set_grid has not been called");
  if (n_edges != ctx->ne) throw lcmg::ArgError("n_edges must equal n_h (n_v - 1) + (n_h - 1) n_v");
  if (!d) throw lcmg::ArgError("null weights");
  LCMG_CUDA(cudaSetDevice(ctx->device));
  if (!dev) {
    for (int64_t e = 0; e < n_edges; ++e)
      if (!(d[e] > 0.0) || !std::isfinite(d[e])) throw lcmg::ArgError("weights must be positive and finite");
    lcmg::copy_sync(ctx->stream, ctx->d.need(n_edges), d, sizeof(double) * n_edges, cudaMemcpyHostToDevice);
  } else {
    LCMG_CUDA(cudaMemcpyAsync(ctx->d.need(n_edges), d, sizeof(double) * n_edges, cudaMemcpyDeviceToDevice,
                              ctx->stream));
  }
  lcmg::refresh_fine(*ctx);
  if (ctx->fwd) lcmg::build_hierarchy(*ctx);
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
}

int lcmg_set_weights(lcmg_ctx* ctx, const double* d, int64_t n_edges) {
  API_BEGIN
  NEED_CTX();
  set_weights_common(ctx, d, n_edges, false);
  API_END
}

int lcmg_set_weights_dev(lcmg_ctx* ctx, const double* d_dev, int64_t n_edges) {
  API_BEGIN
  NEED_CTX();
  set_weights_common(ctx, d_dev, n_edges, true);
  API_END
}

int lcmg_get_weights(lcmg_ctx* ctx, double* d_out, int64_t n_edges) {
  API_BEGIN
  NEED_CTX();
  if (n_edges != ctx->ne || !d_out) throw lcmg::ArgError("bad output buffer");
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  lcmg::copy_sync(ctx->stream, d_out, ctx->d.p, sizeof(double) * n_edges, cudaMemcpyDeviceToHost);
  API_END
}

int lcmg_solve_dev(lcmg_ctx* ctx, int32_t n_lambda, const double* lambda, int32_t n_rhs, const double* b_dev,
                   const double* x0_dev, double* x_dev, double* resid_norm_dev, double* seminorm_dev,
                   int32_t* iters_dev, int32_t* status_dev) {
  API_BEGIN
  NEED_CTX();
  lcmg::StatsScope stats_scope(*ctx);
  LCMG_CUDA(cudaSetDevice(ctx->device));
  lcmg::require_ready(*ctx);
  lcmg::check_lambdas(n_lambda, lambda);
  if (n_rhs < 1 || !b_dev || !x_dev) throw lcmg::ArgError("bad right-hand sides or output");
  lcmg::upload_b(*ctx, n_rhs, b_dev, true);
  const int total = n_lambda * n_rhs;
  std::vector<double> rho(total), eta(total);
  std::vector<int> its(total), st(total);
  const double* x0 = x0_dev;
  lcmg::DevBuf<double>& x0copy = ctx->stage_x0;
  if (x0_dev && x0_dev == x_dev) {  // in-place warm start
    x0copy.need((size_t)total * ctx->n);
    LCMG_CUDA(cudaMemcpyAsync(x0copy.p, x0_dev, sizeof(double) * total * ctx->n, cudaMemcpyDeviceToDevice,
                              ctx->stream));
    x0 = x0copy.p;
  }
  lcmg::solve_all(*ctx, n_lambda, lambda, n_rhs, x0, x_dev, rho.data(), eta.data(), its.data(), st.data());
  if (resid_norm_dev)
    LCMG_CUDA(cudaMemcpyAsync(resid_norm_dev, rho.data(), sizeof(double) * total, cudaMemcpyHostToDevice, ctx->stream));
  if (seminorm_dev)
    LCMG_CUDA(cudaMemcpyAsync(seminorm_dev, eta.data(), sizeof(double) * total, cudaMemcpyHostToDevice, ctx->stream));
  if (iters_dev)
    LCMG_CUDA(cudaMemcpyAsync(iters_dev, its.data(), sizeof(int) * total, cudaMemcpyHostToDevice, ctx->stream));
  if (status_dev)
    LCMG_CUDA(cudaMemcpyAsync(status_dev, st.data(), sizeof(int) * total, cudaMemcpyHostToDevice, ctx->stream));
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  API_END
}

int lcmg_solve(lcmg_ctx* ctx, int32_t n_lambda, const double* lambda, int32_t n_rhs, const double* b,
               const double* x0, double* x, double* resid_norm, double* seminorm, int32_t* iters,
               int32_t* status) {
  API_BEGIN
  NEED_CTX();
  lcmg::StatsScope stats_scope(*ctx);
  LCMG_CUDA(cudaSetDevice(ctx->device));
  lcmg::require_ready(*ctx);
  lcmg::check_lambdas(n_lambda, lambda);
  if (n_rhs < 1 || !b || !x) throw lcmg::ArgError("bad right-hand sides or output");
  const int total = n_lambda * n_rhs;
  lcmg::upload_b(*ctx, n_rhs, b, false);
  lcmg::DevBuf<double>& xd = ctx->stage_x;
  lcmg::DevBuf<double>& x0d = ctx->stage_x0;
  xd.need((size_t)total * ctx->n);
  if (x0) {
    x0d.need((size_t)total * ctx->n);
    lcmg::copy_sync(ctx->stream, x0d.p, x0, sizeof(double) * total * ctx->n, cudaMemcpyHostToDevice);
  }
  lcmg::solve_all(*ctx, n_lambda, lambda, n_rhs, x0 ? x0d.p : nullptr, xd.p, resid_norm, seminorm, iters, status);
  LCMG_CUDA(cudaMemcpyAsync(x, xd.p, sizeof(double) * total * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  API_END
}

int lcmg_lcurve_corner(int32_t k, const double* rho, const double* eta, int32_t* idx) {
  API_BEGIN
  if (k < 3 || !rho || !eta || !idx) throw lcmg::ArgError("the corner needs at least three points");
  for (int i = 0; i < k; ++i)
    if (!(rho[i] > 0) || !(eta[i] > 0) || !std::isfinite(rho[i]) || !std::isfinite(eta[i]))
      throw lcmg::ArgError("rho and eta must be positive and finite");
  *idx = lcmg::corner_host(k, rho, eta);
  API_END
}

int lcmg_cull_lambdas(int32_t m, int32_t i_prev, int32_t* lo, int32_t* hi) {
  API_BEGIN
  if (m < 1 || i_prev < 0 || i_prev > m || !lo || !hi) throw lcmg::ArgError("bad window arguments");
  lcmg::window(m, i_prev, lo, hi);
  API_END
}

namespace lcmg {
// a square CSR matrix from the caller, checked: rows sorted, columns in range
static HostCsr host_square_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* v) {
  if (n < 1 || n > 2147483647LL || !rp || !ci || !v) throw ArgError("bad matrix arguments");
  if (rp[0] != 0) throw ArgError("row_ptr[0] must be 0");
  for (int64_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) throw ArgError("row_ptr must not decrease");
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < 0 || ci[k] >= n) throw ArgError("column index out of range");
      if (k > rp[i] && ci[k] <= ci[k - 1]) throw ArgError("columns must increase within each row");
    }
  }
  HostCsr K;
  K.rows = K.cols = n;
  K.rp.assign(rp, rp + n + 1);
  K.ci.assign(ci, ci + rp[n]);
  K.v.assign(v, v + rp[n]);
  return K;
}
}  // namespace lcmg

int lcmg_rs_split(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, double theta,
                  int8_t* cf) {
  API_BEGIN
  if (!cf || !(theta > 0.0 && theta < 1.0)) throw lcmg::ArgError("null cf or theta outside (0, 1)");
  const lcmg::HostCsr K = lcmg::host_square_csr(n, row_ptr, col, val);
  const std::vector<int8_t> s = lcmg::amg::split(lcmg::amg::strength(K, theta), n);
  std::copy(s.begin(), s.end(), cf);
  API_END
}

int lcmg_rs_interp(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, double theta,
                   const int8_t* cf, int64_t cap, int64_t* p_row_ptr, int32_t* p_col, double* p_val, int64_t* nnz) {
  API_BEGIN
  if (!cf || !nnz || !p_row_ptr || (cap > 0 && (!p_col || !p_val)) || !(theta > 0.0 && theta < 1.0))
    throw lcmg::ArgError("null output or theta outside (0, 1)");
  const lcmg::HostCsr K = lcmg::host_square_csr(n, row_ptr, col, val);
  std::vector<int8_t> c(cf, cf + n);
  for (int8_t f : c)
    if (f != lcmg::amg::kC && f != lcmg::amg::kF) throw lcmg::ArgError("cf entries must be 0 or 1");
  const lcmg::amg::Strength S = lcmg::amg::strength(K, theta);
  for (int64_t i = 0; i < n; ++i) {  // every F point needs a strong C connection
    if (c[i] != lcmg::amg::kF) continue;
    bool has = false;
    for (int64_t k = S.rp[i]; k < S.rp[i + 1] && !has; ++k) has = c[S.ci[k]] == lcmg::amg::kC;
    if (!has) throw lcmg::ArgError("F point " + std::to_string(i) + " has no strong C connection");
  }
  const lcmg::HostCsr P = lcmg::amg::interpolation(K, S, c);
  *nnz = (int64_t)P.ci.size();
  if (cap < *nnz) throw lcmg::ArgError("cap is smaller than the interpolation's entry count");
  std::copy(P.rp.begin(), P.rp.end(), p_row_ptr);
  std::copy(P.ci.begin(), P.ci.end(), p_col);
  std::copy(P.v.begin(), P.v.end(), p_val);
  API_END
}

int lcmg_pmis_split(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, double theta,
                    uint64_t seed, int8_t* cf) {
  API_BEGIN
  if (!cf || !(theta > 0.0 && theta < 1.0)) throw lcmg::ArgError("null cf or theta outside (0, 1)");
  const lcmg::HostCsr K = lcmg::host_square_csr(n, row_ptr, col, val);
  const std::vector<int8_t> s = lcmg::amg::pmis_split(lcmg::amg::strength(K, theta), n, seed, nullptr);
  std::copy(s.begin(), s.end(), cf);
  API_END
}

int lcmg_amg_levels(lcmg_ctx* ctx, int32_t cap, int64_t* sizes, int32_t* n_levels) {
  API_BEGIN
  NEED_CTX();
  if (!n_levels || (cap > 0 && !sizes)) throw lcmg::ArgError("null output");
  if (!ctx->am_ok) throw std::runtime_error("no classical AMG hierarchy has been built for the current weights");
  *n_levels = (int32_t)ctx->am.size();
  for (int32_t k = 0; k < cap && k < *n_levels; ++k) sizes[k] = ctx->am[k].n;
  API_END
}

int lcmg_update_weights_dev(lcmg_ctx* ctx, const double* x_star_dev, double q, double d_min) {
  API_BEGIN
  NEED_CTX();
  if (ctx->nv == 0 || !x_star_dev) throw lcmg::ArgError("grid not set or null x");
  LCMG_CUDA(cudaSetDevice(ctx->device));
  lcmg::update_weights_dev(*ctx, x_star_dev, q, d_min);
  if (ctx->fwd) lcmg::build_hierarchy(*ctx);
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  API_END
}

int lcmg_update_weights(lcmg_ctx* ctx, const double* x_star, double q, double d_min, double* d_out) {
  API_BEGIN
  NEED_CTX();
  if (ctx->nv == 0 || !x_star) throw lcmg::ArgError("grid not set or null x");
  LCMG_CUDA(cudaSetDevice(ctx->device));
  lcmg::DevBuf<double>& xs = ctx->stage_x;
  xs.need(ctx->n);
  lcmg::copy_sync(ctx->stream, xs.p, x_star, sizeof(double) * ctx->n, cudaMemcpyHostToDevice);
  lcmg::update_weights_dev(*ctx, xs.p, q, d_min);
  if (ctx->fwd) lcmg::build_hierarchy(*ctx);
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (d_out) lcmg::copy_sync(ctx->stream, d_out, ctx->d.p, sizeof(double) * ctx->ne, cudaMemcpyDeviceToHost);
  API_END
}

int lcmg_lcurve_run_dev(lcmg_ctx* ctx, int32_t m_lambda, const double* lambda, const double* b_dev,
                        int32_t max_outer, double* x_out_dev, int32_t* lambda_idx_history, int32_t* n_outer,
                        int64_t* n_solves, int64_t* n_converged) {
  API_BEGIN
  NEED_CTX();
  lcmg::StatsScope stats_scope(*ctx);
  LCMG_CUDA(cudaSetDevice(ctx->device));
  if (!b_dev || !x_out_dev || !lambda_idx_history || !n_outer) throw lcmg::ArgError("null argument");
  lcmg::require_ready(*ctx);
  // Algorithm 2 starts from D = I
  std::vector<double> ones(ctx->ne, 1.0);
  lcmg::copy_sync(ctx->stream, ctx->d.need(ctx->ne), ones.data(), sizeof(double) * ctx->ne, cudaMemcpyHostToDevice);
  lcmg::refresh_fine(*ctx);
  lcmg::build_hierarchy(*ctx);
  lcmg::upload_b(*ctx, 1, b_dev, true);
  lcmg::lcurve_run_impl(*ctx, m_lambda, lambda, max_outer, x_out_dev, lambda_idx_history, n_outer, n_solves,
                        n_converged);
  API_END
}

int lcmg_lcurve_run(lcmg_ctx* ctx, int32_t m_lambda, const double* lambda, const double* b, int32_t max_outer,
                    double* x_out, int32_t* lambda_idx_history, int32_t* n_outer, int64_t* n_solves,
                    int64_t* n_converged) {
  API_BEGIN
  NEED_CTX();
  lcmg::StatsScope stats_scope(*ctx);
  LCMG_CUDA(cudaSetDevice(ctx->device));
  if (!b || !x_out || !lambda_idx_history || !n_outer) throw lcmg::ArgError("null argument");
  lcmg::require_ready(*ctx);
  lcmg::DevBuf<double>& bd = ctx->stage_b;
  lcmg::DevBuf<double>& xd = ctx->stage_x;
  bd.need(ctx->m);
  xd.need(ctx->n);
  lcmg::copy_sync(ctx->stream, bd.p, b, sizeof(double) * ctx->m, cudaMemcpyHostToDevice);
  std::vector<double> ones(ctx->ne, 1.0);
  lcmg::copy_sync(ctx->stream, ctx->d.need(ctx->ne), ones.data(), sizeof(double) * ctx->ne, cudaMemcpyHostToDevice);
  lcmg::refresh_fine(*ctx);
  lcmg::build_hierarchy(*ctx);
  lcmg::upload_b(*ctx, 1, bd.p, true);
  lcmg::lcurve_run_impl(*ctx, m_lambda, lambda, max_outer, xd.p, lambda_idx_history, n_outer, n_solves,
                        n_converged);
  lcmg::copy_sync(ctx->stream, x_out, xd.p, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost);
  API_END
}

int lcmg_get_stats(lcmg_ctx* ctx, lcmg_stats* out) {
  API_BEGIN
  NEED_CTX();
  if (!out) throw lcmg::ArgError("null output");
  *out = ctx->stats;
  API_END
}

int lcmg_apply_normal_dev(lcmg_ctx* ctx, int32_t n_cols, const double* lambda, const double* x_dev,
                          double* y_dev) {
  API_BEGIN
  NEED_CTX();
  LCMG_CUDA(cudaSetDevice(ctx->device));
  lcmg::require_ready(*ctx);
  if (n_cols < 1 || n_cols > lcmg::kMaxB || !lambda || !x_dev || !y_dev) throw lcmg::ArgError("bad arguments");
  const int B = n_cols;
  lcmg::ensure_work(*ctx, B);
  std::vector<double> l2(B);
  for (int j = 0; j < B; ++j) l2[j] = lambda[j] * lambda[j];
  lcmg::copy_sync(ctx->stream, ctx->lam2.p, l2.data(), sizeof(double) * B, cudaMemcpyHostToDevice);
  const int g = lcmg::grid_for(ctx->n, B, ctx->maxblk);
  klaunch(lcmg::k_planar_to_inter, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, ctx->n, B, x_dev, ctx->x64.p);
  LCMG_LAUNCHED();
  LCMG_CUDA(cudaMemsetAsync(ctx->c64.p, 0, sizeof(double) * ctx->n * B, ctx->stream));
  lcmg::Batch<double> b(*ctx, B);
  b.true_residual(ctx->part_x.p);  // r64 = 0 - K x
  const int ge = (int)std::min<int64_t>(((int64_t)ctx->n * B + lcmg::kBlock - 1) / lcmg::kBlock, ctx->maxblk);
  klaunch(lcmg::k_negate, dim3(ge), dim3(lcmg::kBlock), 0, ctx->stream, (int64_t)ctx->n * B, ctx->r64.p);
  LCMG_LAUNCHED();
  klaunch(lcmg::k_inter_to_planar, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, ctx->n, B, ctx->r64.p, y_dev);
  LCMG_LAUNCHED();
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  API_END
}

int lcmg_apply_vcycle_dev(lcmg_ctx* ctx, int32_t n_cols, const double* lambda, const double* r_dev,
                          double* z_dev) {
  API_BEGIN
  NEED_CTX();
  LCMG_CUDA(cudaSetDevice(ctx->device));
  lcmg::require_ready(*ctx);
  if (n_cols < 1 || n_cols > lcmg::kMaxB || !lambda || !r_dev || !z_dev) throw lcmg::ArgError("bad arguments");
  const int B = n_cols;
  lcmg::ensure_work(*ctx, B);
  std::vector<double> lam(lambda, lambda + B);
  if (ctx->prm.precond == 1) {  // the paper's V(2,1), one column at a time, FP64
    lcmg::pm_build(*ctx);
    lcmg::PaperMG pmg(*ctx);
    pmg.L = pmg.amg ? (int)ctx->am.size() : (int)ctx->lev.size();
    for (int j = 0; j < B; ++j) {
      pmg.setup(lam[j]);
      pmg.cycle(0, r_dev + (int64_t)j * ctx->n, z_dev + (int64_t)j * ctx->n);
    }
    LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
    return LCMG_OK;
  }
  const int g = lcmg::grid_for(ctx->n, B, ctx->maxblk);
  if (ctx->prm.precision == LCMG_PREC_FP64) {
    lcmg::Batch<double> b(*ctx, B);
    b.setup(lam);
    klaunch(lcmg::k_planar_to_inter, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, ctx->n, B, r_dev, reinterpret_cast<double*>(ctx->r.p));
    LCMG_LAUNCHED();
    b.vcycle(reinterpret_cast<double*>(ctx->r.p), reinterpret_cast<double*>(ctx->z.p), ctx->part_x.p);
    klaunch(lcmg::k_inter_to_planar, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, ctx->n, B, reinterpret_cast<double*>(ctx->z.p), z_dev);
    LCMG_LAUNCHED();
  } else {
    lcmg::Batch<float> b(*ctx, B);
    b.setup(lam);
    klaunch(lcmg::k_planar_to_inter, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, ctx->n, B, r_dev, ctx->r64.p);
    LCMG_LAUNCHED();
    klaunch(lcmg::k_convert<double, float>, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, (int64_t)ctx->n * B, ctx->r64.p,
                                                                         reinterpret_cast<float*>(ctx->r.p));
    LCMG_LAUNCHED();
    b.vcycle(reinterpret_cast<float*>(ctx->r.p), reinterpret_cast<float*>(ctx->z.p), ctx->part_x.p);
    klaunch(lcmg::k_convert<float, double>, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, (int64_t)ctx->n * B,
                                                                         reinterpret_cast<float*>(ctx->z.p), ctx->r64.p);
    LCMG_LAUNCHED();
    klaunch(lcmg::k_inter_to_planar, dim3(g), dim3(lcmg::kBlock), 0, ctx->stream, ctx->n, B, ctx->r64.p, z_dev);
    LCMG_LAUNCHED();
  }
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  API_END
}

int lcmg_get_level(lcmg_ctx* ctx, int32_t k, int32_t* n_v, int32_t* n_h, double* gl, double* ga) {
  API_BEGIN
  NEED_CTX();
  lcmg::require_ready(*ctx);
  if (k < 0 || k >= (int)ctx->lev.size()) throw lcmg::ArgError("level out of range");
  const lcmg::Level& L = ctx->lev[k];
  if (n_v) *n_v = L.nv;
  if (n_h) *n_h = L.nh;
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (k > 0) {
    if (gl) lcmg::copy_sync(ctx->stream, gl, L.gl.p, sizeof(double) * lcmg::kStencil * L.n, cudaMemcpyDeviceToHost);
    if (ga) lcmg::copy_sync(ctx->stream, ga, L.ga.p, sizeof(double) * lcmg::kStencil * L.n, cudaMemcpyDeviceToHost);
  }
  API_END
}

int lcmg_num_levels(lcmg_ctx* ctx, int32_t* levels) {
  API_BEGIN
  NEED_CTX();
  lcmg::require_ready(*ctx);
  if (!levels) throw lcmg::ArgError("null output");
  *levels = (int)ctx->lev.size();
  API_END
}

int lcmg_get_diag(lcmg_ctx* ctx, double* diag_out) {
  API_BEGIN
  NEED_CTX();
  if (ctx->fwd == 0 || !diag_out) throw lcmg::ArgError("forward operator not set or null output");
  LCMG_CUDA(cudaStreamSynchronize(ctx->stream));
  lcmg::copy_sync(ctx->stream, diag_out, ctx->diag.p, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost);
  API_END
}

}  // extern "C"
