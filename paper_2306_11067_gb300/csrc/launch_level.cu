// Launchers of the V-cycle level kernels, the coarsest-level dense setup,
// the Galerkin products and the PCG vector updates.
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "launch.h"
#include "vcoarse.cuh"
#include "vtail.cuh"
#include "vfine.cuh"
#include "vfused.cuh"

namespace lcmg {

template <class T>
void launch_dinv(const LevelView<T>& L, int B, const double* lam2, int smoother, double omega,
                 T* dinv, int max_blocks, cudaStream_t s) {
  const int g = grid_for(L.n, B, max_blocks);
  if constexpr (std::is_same<T, float>::value) {
    if (L.h16) {
      if (L.fine)
        klaunch(k_dinv<FineOpH, float>, dim3(g), dim3(kBlock), 0, s, L.fh, L.n, B, lam2, smoother, omega, dinv);
      else
        klaunch(k_dinv<CoarseOpH, float>, dim3(g), dim3(kBlock), 0, s, L.ch, L.n, B, lam2, smoother, omega, dinv);
      LCMG_LAUNCHED();
      return;
    }
  }
  if (L.fine)
    klaunch(k_dinv<FineOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.fine_op(), L.n, B, lam2, smoother, omega, dinv);
  else
    klaunch(k_dinv<CoarseOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.coarse_op(), L.n, B, lam2, smoother, omega, dinv);
  LCMG_LAUNCHED();
}

template <class T>
void launch_smooth_zero(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r,
                        T* z, int two, int max_blocks, cudaStream_t s) {
  const int g = grid_for(L.n, B, max_blocks);
  if (L.fine)
    klaunch(k_smooth_zero<FineOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.fine_op(), L.n, B, lam2, dinv, r, z, two);
  else
    klaunch(k_smooth_zero<CoarseOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.coarse_op(), L.n, B, lam2, dinv, r, z, two);
  LCMG_LAUNCHED();
}

template <class T>
int launch_smooth(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r,
                  const T* zin, T* zout, const int* active, double* part, int max_blocks,
                  cudaStream_t s) {
  const int g = grid_for(L.n, B, max_blocks);
  if (L.fine)
    klaunch(k_smooth<FineOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.fine_op(), L.n, B, lam2, dinv, r, zin, zout, active, part);
  else
    klaunch(k_smooth<CoarseOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.coarse_op(), L.n, B, lam2, dinv, r, zin, zout, active, part);
  LCMG_LAUNCHED();
  return g;
}

template <class T>
void launch_residual(const LevelView<T>& L, int B, const T* lam2, const T* r, const T* z, T* res,
                     int max_blocks, cudaStream_t s) {
  const int g = grid_for(L.n, B, max_blocks);
  if (L.fine)
    klaunch(k_residual<FineOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.fine_op(), L.n, B, lam2, r, z, res);
  else
    klaunch(k_residual<CoarseOp<T>, T>, dim3(g), dim3(kBlock), 0, s, L.coarse_op(), L.n, B, lam2, r, z, res);
  LCMG_LAUNCHED();
}

// Grid of a tile kernel: every tile once, at most the blocks resident at
// once on the device and at most kMaxTileBlocks (rows of the partial sums).
template <class K>
static int tile_grid(K kern, int threads, int ntiles, size_t smem = 0) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  LCMG_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_pair(reinterpret_cast<const void*>(kern), dev);
  int wave;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
      int nb = 0, sms = 0;
      LCMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem));
      LCMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      it = cache.emplace(key, std::max(1, nb) * sms).first;
    }
    wave = it->second;
  }
  return std::max(1, std::min(std::min(ntiles, wave), kMaxTileBlocks));
}

template <class Op, class T, int NU>
static int vdown_one(const Op& op, int B, const T* lam2, const T* dinv, const T* r, T* zpre, T* rc, int ntx,
                     int ntiles, cudaStream_t s) {
  auto k = k_vdown<Op, T, NU>;
  const int g = tile_grid(k, vtile_threads<Op, T, NU>(), ntiles);
  klaunch(k, dim3((unsigned)g, (unsigned)B), dim3(vtile_threads<Op, T, NU>()), 0, s, op, B, lam2, dinv, r, zpre, rc,
          ntx, ntiles);
  return g;
}

template <class Op, class T, int NU>
static int vup_one(const Op& op, int B, const T* lam2, const T* dinv, const T* r, const T* ec, const T* zpre,
                   T* zout, double* part, int ntx, int ntiles, cudaStream_t s) {
  auto k = k_vup<Op, T, NU>;
  const int g = tile_grid(k, vtile_threads<Op, T, NU>(), ntiles);
  klaunch(k, dim3((unsigned)g, (unsigned)B), dim3(vtile_threads<Op, T, NU>()), 0, s, op, B, lam2, dinv, r, ec, zpre,
          zout, ntx, ntiles, part);
  return g;
}

// FP16 coarse levels with one sweep: the staged, double-buffered tile kernels
static int vdown_h(const CoarseOpH& op, int B, const float* dinv, const float* r, float* zpre, float* rc, int ntx,
                   int ntiles, cudaStream_t s) {
  const size_t smem = 2 * sizeof(VcDownStage);
  const int g = tile_grid(k_vdown_h, kVcThreads, ntiles, smem);
  klaunch(k_vdown_h, dim3((unsigned)g, (unsigned)B), dim3(kVcThreads), smem, s, op, B, dinv, r, zpre, rc, ntx,
          ntiles);
  return g;
}
static int vup_h(const CoarseOpH& op, int B, const float* dinv, const float* r, const float* ec, const float* zpre,
                 float* zout, double* part, int ntx, int ntiles, cudaStream_t s) {
  const size_t smem = 2 * sizeof(VcUpStage);
  const int g = tile_grid(k_vup_h, kVcThreads, ntiles, smem);
  klaunch(k_vup_h, dim3((unsigned)g, (unsigned)B), dim3(kVcThreads), smem, s, op, B, dinv, r, ec, zpre, zout, ntx,
          ntiles, part);
  return g;
}

template <class T>
int launch_vdown(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r, T* zpre, T* rc,
                 int nu, cudaStream_t s) {
  const int ntx = (L.nv / 2 + kVTile - 1) / kVTile, nty = (L.nh / 2 + kVTile - 1) / kVTile;
  const int nt = ntx * nty;
  int g;
  if constexpr (std::is_same<T, float>::value) {
    if (L.h16) {
      if (L.fine)
        g = nu == 1 ? vdown_one<FineOpH, float, 1>(L.fh, B, lam2, dinv, r, zpre, rc, ntx, nt, s)
                    : vdown_one<FineOpH, float, 2>(L.fh, B, lam2, dinv, r, zpre, rc, ntx, nt, s);
      else
        g = nu == 1 ? vdown_h(L.ch, B, dinv, r, zpre, rc, ntx, nt, s)
                    : vdown_one<CoarseOpH, float, 2>(L.ch, B, lam2, dinv, r, zpre, rc, ntx, nt, s);
      LCMG_LAUNCHED();
      return g;
    }
  }
  if (L.fine)
    g = nu == 1 ? vdown_one<FineOp<T>, T, 1>(L.fine_op(), B, lam2, dinv, r, zpre, rc, ntx, nt, s)
                : vdown_one<FineOp<T>, T, 2>(L.fine_op(), B, lam2, dinv, r, zpre, rc, ntx, nt, s);
  else
    g = nu == 1 ? vdown_one<CoarseOp<T>, T, 1>(L.coarse_op(), B, lam2, dinv, r, zpre, rc, ntx, nt, s)
                : vdown_one<CoarseOp<T>, T, 2>(L.coarse_op(), B, lam2, dinv, r, zpre, rc, ntx, nt, s);
  LCMG_LAUNCHED();
  return g;
}

template <class T>
int launch_vup(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r, const T* ec,
               const T* zpre, T* zout, double* part, int nu, cudaStream_t s) {
  const int ntx = (L.nv / 2 + kVTile - 1) / kVTile, nty = (L.nh / 2 + kVTile - 1) / kVTile;
  const int nt = ntx * nty;
  int g;
  if constexpr (std::is_same<T, float>::value) {
    if (L.h16) {
      if (L.fine)
        g = nu == 1 ? vup_one<FineOpH, float, 1>(L.fh, B, lam2, dinv, r, ec, zpre, zout, part, ntx, nt, s)
                    : vup_one<FineOpH, float, 2>(L.fh, B, lam2, dinv, r, ec, zpre, zout, part, ntx, nt, s);
      else
        g = nu == 1 ? vup_h(L.ch, B, dinv, r, ec, zpre, zout, part, ntx, nt, s)
                    : vup_one<CoarseOpH, float, 2>(L.ch, B, lam2, dinv, r, ec, zpre, zout, part, ntx, nt, s);
      LCMG_LAUNCHED();
      return g;
    }
  }
  if (L.fine)
    g = nu == 1 ? vup_one<FineOp<T>, T, 1>(L.fine_op(), B, lam2, dinv, r, ec, zpre, zout, part, ntx, nt, s)
                : vup_one<FineOp<T>, T, 2>(L.fine_op(), B, lam2, dinv, r, ec, zpre, zout, part, ntx, nt, s);
  else
    g = nu == 1 ? vup_one<CoarseOp<T>, T, 1>(L.coarse_op(), B, lam2, dinv, r, ec, zpre, zout, part, ntx, nt, s)
                : vup_one<CoarseOp<T>, T, 2>(L.coarse_op(), B, lam2, dinv, r, ec, zpre, zout, part, ntx, nt, s);
  LCMG_LAUNCHED();
  return g;
}

bool vtail_fits(int nlev) { return nlev >= 2 && nlev <= kTailMaxLevels; }

void launch_vtail(const TailLevelIn* levels, int nlev, const double* kinv, int nc, int B, cudaStream_t s) {
  if (!vtail_fits(nlev)) throw ArgError("tail of the V-cycle: level count out of range");
  TailArgs a{};
  a.nlev = nlev;
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off += (bytes + 15) / 16 * 16;
    return o;
  };
  for (int k = 0; k < nlev; ++k) {
    const TailLevelIn& in = levels[k];
    const int n = in.op.nv * in.op.nh;
    TailLevel& L = a.lv[k];
    L.op = in.op;
    L.dinv = in.dinv;
    L.rhs = in.rhs;
    L.z = in.z;
    const bool coarsest = k == nlev - 1;
    L.o_rows = coarsest ? 0 : take(48 * n);
    L.o_s = coarsest ? 0 : take(4 * n);
    L.o_d = coarsest ? 0 : take(4 * n);
    L.o_r = take(4 * n);
    L.o_t = coarsest ? 0 : take(4 * n);
    L.o_res = coarsest ? 0 : take(4 * n);
    L.o_z = take(4 * n);
  }
  a.kinv = kinv;
  a.nc = nc;
  static int optin_dev = -1;
  int dev = 0;
  LCMG_CUDA(cudaGetDevice(&dev));
  if (optin_dev != dev) {
    int maxsm = 0;
    LCMG_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    LCMG_CUDA(cudaFuncSetAttribute(k_vtail_h, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    optin_dev = dev;
  }
  klaunch(k_vtail_h, dim3(1, (unsigned)B), dim3(kTailThreads), (size_t)off, s, a, B);
  LCMG_LAUNCHED();
}

// Grid of the fused one-column updates: every block re-sums the partials of
// the dot products it needs (FP64), so the grid stays at 4 blocks of 256
// threads per SM (a full SM of resident warps streams the vectors)
static int fused_update_grid(int64_t n, int max_blocks) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    LCMG_CUDA(cudaGetDevice(&dev));
    LCMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return std::min(grid_for(n, 1, max_blocks), std::max(1, 4 * sms));
}

// Rows per strip of the row-streaming kernels: at most `most`, and few
// enough that the strips number about four warps per SM slot of a wave
// (one warp walks a strip in sequence, so on a small grid long strips leave
// most of the GPU idle), but at least `least` (the strip's halo rows are
// computed twice).
static int strip_rows(int nsi, int len, int most, int least) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    LCMG_CUDA(cudaGetDevice(&dev));
    LCMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t want = (int64_t)sms * 32;  // warps resident at 4 blocks of 8 warps per SM
  const int64_t per_col = std::max<int64_t>(1, (want + nsi - 1) / nsi);  // strips wanted along the rows
  const int rows = (int)((len + per_col - 1) / per_col);
  return std::max(least, std::min(most, rows));
}

int launch_vfine_down(const LevelView<float>& L, int B, const float* lam2, int smoother, double omega,
                      const float* r, float* rc, cudaStream_t s) {
  const int nt = ((L.nv + kFineTI - 1) / kFineTI) * ((L.nh + kFineTJ - 1) / kFineTJ);
  int g;
  if (L.h16 && L.nv % 2 == 0 && L.nh % 2 == 0 && (int64_t)L.nv * L.nh * B < (int64_t(1) << 31)) {  // row streaming
    const int nsi = (L.nv / 2 + kDownCols - 1) / kDownCols;
    const int crows = strip_rows(nsi, L.nh / 2, kStripCoarse, 2);
    const int nst = nsi * ((L.nh / 2 + crows - 1) / crows);
    auto k = B == 1 ? k_vfine_down_s<true> : k_vfine_down_s<false>;
    g = tile_grid(k, kFineThreads, (nst + kFineThreads / 32 - 1) / (kFineThreads / 32));
    klaunch(k, dim3((unsigned)g, (unsigned)B), dim3(kFineThreads), 0, s, L.fh, B, lam2, smoother, (float)omega, r,
            rc, nsi, nst, crows);
  } else if (L.h16) {
    g = tile_grid(k_vfine_down<FineOpH>, kFineThreads, nt);
    klaunch(k_vfine_down<FineOpH>, dim3((unsigned)g, (unsigned)B), dim3(kFineThreads), 0, s, L.fh, B, lam2, smoother,
            (float)omega, r, rc, nt);
  } else {
    g = tile_grid(k_vfine_down<FineOp<float>>, kFineThreads, nt);
    klaunch(k_vfine_down<FineOp<float>>, dim3((unsigned)g, (unsigned)B), dim3(kFineThreads), 0, s, L.fine_op(), B,
            lam2, smoother, (float)omega, r, rc, nt);
  }
  LCMG_LAUNCHED();
  return g;
}

int launch_vfine_up(const LevelView<float>& L, int B, const float* lam2, int smoother, double omega,
                    const float* r, const float* ec, float* zout, double* part, cudaStream_t s) {
  const int nt = ((L.nv + kFineTI - 1) / kFineTI) * ((L.nh + kFineTJ - 1) / kFineTJ);
  int g;
  if (L.h16 && L.nv % 2 == 0 && L.nh % 2 == 0 && (int64_t)L.nv * L.nh * B < (int64_t(1) << 31)) {  // row streaming
    const int nsi = (L.nv + kUpCols - 1) / kUpCols;
    const int rows = strip_rows(nsi, L.nh, kStripRows, 4);
    const int nst = nsi * ((L.nh + rows - 1) / rows);
    auto k = B == 1 ? k_vfine_up_s<true> : k_vfine_up_s<false>;
    g = tile_grid(k, kFineThreads, (nst + kFineThreads / 32 - 1) / (kFineThreads / 32));
    klaunch(k, dim3((unsigned)g, (unsigned)B), dim3(kFineThreads), 0, s, L.fh, B, lam2, smoother, (float)omega, r,
            ec, zout, nsi, nst, rows, part);
  } else if (L.h16) {
    g = tile_grid(k_vfine_up<FineOpH>, kFineThreads, nt);
    klaunch(k_vfine_up<FineOpH>, dim3((unsigned)g, (unsigned)B), dim3(kFineThreads), 0, s, L.fh, B, lam2, smoother,
            (float)omega, r, ec, zout, nt, part);
  } else {
    g = tile_grid(k_vfine_up<FineOp<float>>, kFineThreads, nt);
    klaunch(k_vfine_up<FineOp<float>>, dim3((unsigned)g, (unsigned)B), dim3(kFineThreads), 0, s, L.fine_op(), B,
            lam2, smoother, (float)omega, r, ec, zout, nt, part);
  }
  LCMG_LAUNCHED();
  return g;
}

template <class T>
void launch_restrict(int nvc, int nhc, int B, const T* rf, T* rc, int max_blocks, cudaStream_t s) {
  const int g = grid_for((int64_t)nvc * nhc, B, max_blocks);
  klaunch(k_restrict<T>, dim3(g), dim3(kBlock), 0, s, nvc, nhc, B, rf, rc);
  LCMG_LAUNCHED();
}

template <class T>
void launch_prolong_add(int nvc, int nhc, int B, const T* ec, T* zf, int max_blocks, cudaStream_t s) {
  const int g = grid_for((int64_t)4 * nvc * nhc, B, max_blocks);
  klaunch(k_prolong_add<T>, dim3(g), dim3(kBlock), 0, s, nvc, nhc, B, ec, zf);
  LCMG_LAUNCHED();
}

template <class T>
void launch_coarse_solve(int nc, int B, const double* kinv, const T* rc, T* ec, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)nc;
  dim3 grid((unsigned)((nc + kBlock / 32 - 1) / (kBlock / 32)), (unsigned)B);
  klaunch(k_coarse_solve<T>, dim3(grid), dim3(kBlock), smem, s, nc, B, kinv, rc, ec);
  LCMG_LAUNCHED();
}

void launch_dense_setup(const LevelView<double>& L, int B, const double* lam2, double* M, double* W,
                        double* K, int* info, int max_blocks, cudaStream_t s) {
  const int64_t nc = L.n;
  LCMG_CUDA(cudaMemsetAsync(M, 0, sizeof(double) * (size_t)B * nc * nc, s));
  const int g = grid_for(nc, B, max_blocks);
  if (L.fine)
    klaunch(k_dense_assemble<FineOp<double>>, dim3(g), dim3(kBlock), 0, s, L.fine_op(), nc, B, lam2, M);
  else
    klaunch(k_dense_assemble<CoarseOp<double>>, dim3(g), dim3(kBlock), 0, s, L.coarse_op(), nc, B, lam2, M);
  LCMG_LAUNCHED();
  klaunch(k_cholesky_inverse, dim3(B), dim3(kBlock), 0, s, (int)nc, M, W, K, info);
  LCMG_LAUNCHED();
}

void launch_galerkin(const RapIn& in, int nvc, int nhc, double* out, int max_blocks, cudaStream_t s) {
  const int64_t work = (int64_t)nvc * nhc * kStencil;
  int64_t g = (work + kBlock - 1) / kBlock;
  if (g > max_blocks) g = max_blocks;
  klaunch(k_galerkin, dim3((unsigned)g), dim3(kBlock), 0, s, in, nvc, nhc, out);
  LCMG_LAUNCHED();
}

template <class T, class TX>
int launch_update_xr(int64_t n, int B, const ColState& st, const T* p, const T* q, TX* x, T* r,
                     double* part, int max_blocks, cudaStream_t s) {
  const int g = grid_for(n, B, max_blocks);
  klaunch(k_update_xr<T, TX>, dim3(g), dim3(kBlock), 0, s, n, B, st, p, q, x, r, part);
  LCMG_LAUNCHED();
  return g;
}

template <class T, class TX>
int launch_update_xr_alpha(int64_t n, const ColState& st, int nb_pq, const double* pq_part, const T* p,
                           const T* q, TX* x, T* r, double* part, int max_blocks, cudaStream_t s) {
  const int g = fused_update_grid(n, max_blocks);
  klaunch(k_update_xr_alpha<T, TX>, dim3(g), dim3(kBlock), 0, s, n, st, nb_pq, pq_part, p, q, x, r, part);
  LCMG_LAUNCHED();
  return g;
}

template <class T>
void launch_update_p_beta(int64_t n, const ColState& st, int nb_rr, const double* rr_part, int nb_rz,
                          const double* rz_part, int maxit, double rel_trigger, const T* z, T* p, int max_blocks,
                          cudaStream_t s) {
  const int g = fused_update_grid(n, max_blocks);
  klaunch(k_update_p_beta<T>, dim3(g), dim3(kBlock), 0, s, n, st, nb_rr, rr_part, nb_rz, rz_part, maxit, rel_trigger,
          z, p);
  LCMG_LAUNCHED();
}

template <class T>
void launch_update_p(int64_t n, int B, const ColState& st, const T* z, T* p, int max_blocks,
                     cudaStream_t s) {
  const int g = grid_for(n, B, max_blocks);
  klaunch(k_update_p<T>, dim3(g), dim3(kBlock), 0, s, n, B, st, z, p);
  LCMG_LAUNCHED();
}

template <class T>
void launch_copy_cols(int64_t n, int B, const int* flag, const T* src, T* dst, int max_blocks,
                      cudaStream_t s) {
  const int g = grid_for(n, B, max_blocks);
  klaunch(k_copy_cols<T>, dim3(g), dim3(kBlock), 0, s, n, B, flag, src, dst);
  LCMG_LAUNCHED();
}

#define LCMG_INST_T(T)                                                                          \
  template void launch_dinv<T>(const LevelView<T>&, int, const double*, int, double, T*, int,   \
                               cudaStream_t);                                                   \
  template void launch_smooth_zero<T>(const LevelView<T>&, int, const T*, const T*, const T*,   \
                                      T*, int, int, cudaStream_t);                              \
  template int launch_smooth<T>(const LevelView<T>&, int, const T*, const T*, const T*,         \
                                const T*, T*, const int*, double*, int, cudaStream_t);          \
  template void launch_residual<T>(const LevelView<T>&, int, const T*, const T*, const T*, T*,  \
                                   int, cudaStream_t);                                          \
  template void launch_restrict<T>(int, int, int, const T*, T*, int, cudaStream_t);             \
  template int launch_vdown<T>(const LevelView<T>&, int, const T*, const T*, const T*, T*, T*,    \
                               int, cudaStream_t);                                                \
  template int launch_vup<T>(const LevelView<T>&, int, const T*, const T*, const T*, const T*,    \
                             const T*, T*, double*, int, cudaStream_t);                           \
  template void launch_prolong_add<T>(int, int, int, const T*, T*, int, cudaStream_t);          \
  template void launch_coarse_solve<T>(int, int, const double*, const T*, T*, cudaStream_t);    \
  template void launch_update_p<T>(int64_t, int, const ColState&, const T*, T*, int,            \
                                   cudaStream_t);                                               \
  template void launch_copy_cols<T>(int64_t, int, const int*, const T*, T*, int, cudaStream_t);       \
  template void launch_update_p_beta<T>(int64_t, const ColState&, int, const double*, int, const double*, int, \
                                        double, const T*, T*, int, cudaStream_t);
LCMG_INST_T(float)
LCMG_INST_T(double)
#undef LCMG_INST_T
template int launch_update_xr<double, double>(int64_t, int, const ColState&, const double*,
                                              const double*, double*, double*, double*, int,
                                              cudaStream_t);
template int launch_update_xr<float, float>(int64_t, int, const ColState&, const float*,
                                            const float*, float*, float*, double*, int,
                                            cudaStream_t);
template int launch_update_xr_alpha<double, double>(int64_t, const ColState&, int, const double*,
                                                    const double*, const double*, double*, double*,
                                                    double*, int, cudaStream_t);
template int launch_update_xr_alpha<float, float>(int64_t, const ColState&, int, const double*, const float*,
                                                  const float*, float*, float*, double*, int,
                                                  cudaStream_t);

}  // namespace lcmg
