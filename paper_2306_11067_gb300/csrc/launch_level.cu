// Launchers of the V-cycle level kernels, the coarsest-level dense setup,
// the Galerkin products and the PCG vector updates.
#include "launch.h"
#include "vfused.cuh"

namespace lcmg {

template <class T>
void launch_dinv(const LevelView<T>& L, int B, const double* lam2, int smoother, double omega,
                 T* dinv, int max_blocks, cudaStream_t s) {
  const int g = grid_for(L.n, B, max_blocks);
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

template <class T>
int launch_vdown(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r, T* zpre, T* rc,
                 int nu, cudaStream_t s) {
  const int ntx = (L.nv / 2 + kVTile - 1) / kVTile, nty = (L.nh / 2 + kVTile - 1) / kVTile;
  const dim3 grid((unsigned)(ntx * nty), (unsigned)B);
  if (L.fine) {
    if (nu == 1) klaunch(k_vdown<FineOp<T>, T, 1>, grid, dim3(vtile_threads<FineOp<T>, T, 1>()), 0, s, L.fine_op(), B, lam2, dinv, r, zpre, rc, ntx);
    else klaunch(k_vdown<FineOp<T>, T, 2>, grid, dim3(vtile_threads<FineOp<T>, T, 2>()), 0, s, L.fine_op(), B, lam2, dinv, r, zpre, rc, ntx);
  } else {
    if (nu == 1) klaunch(k_vdown<CoarseOp<T>, T, 1>, grid, dim3(vtile_threads<CoarseOp<T>, T, 1>()), 0, s, L.coarse_op(), B, lam2, dinv, r, zpre, rc, ntx);
    else klaunch(k_vdown<CoarseOp<T>, T, 2>, grid, dim3(vtile_threads<CoarseOp<T>, T, 2>()), 0, s, L.coarse_op(), B, lam2, dinv, r, zpre, rc, ntx);
  }
  LCMG_LAUNCHED();
  return ntx * nty;
}

template <class T>
int launch_vup(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r, const T* ec,
               const T* zpre, T* zout, double* part, int nu, cudaStream_t s) {
  const int ntx = (L.nv / 2 + kVTile - 1) / kVTile, nty = (L.nh / 2 + kVTile - 1) / kVTile;
  const dim3 grid((unsigned)(ntx * nty), (unsigned)B);
  if (L.fine) {
    if (nu == 1) klaunch(k_vup<FineOp<T>, T, 1>, grid, dim3(vtile_threads<FineOp<T>, T, 1>()), 0, s, L.fine_op(), B, lam2, dinv, r, ec, zpre, zout, ntx, part);
    else klaunch(k_vup<FineOp<T>, T, 2>, grid, dim3(vtile_threads<FineOp<T>, T, 2>()), 0, s, L.fine_op(), B, lam2, dinv, r, ec, zpre, zout, ntx, part);
  } else {
    if (nu == 1) klaunch(k_vup<CoarseOp<T>, T, 1>, grid, dim3(vtile_threads<CoarseOp<T>, T, 1>()), 0, s, L.coarse_op(), B, lam2, dinv, r, ec, zpre, zout, ntx, part);
    else klaunch(k_vup<CoarseOp<T>, T, 2>, grid, dim3(vtile_threads<CoarseOp<T>, T, 2>()), 0, s, L.coarse_op(), B, lam2, dinv, r, ec, zpre, zout, ntx, part);
  }
  LCMG_LAUNCHED();
  return ntx * nty;
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
  const int g = grid_for(n, 1, max_blocks);
  klaunch(k_update_xr_alpha<T, TX>, dim3(g), dim3(kBlock), 0, s, n, st, nb_pq, pq_part, p, q, x, r, part);
  LCMG_LAUNCHED();
  return g;
}

template <class T>
void launch_update_p_beta(int64_t n, const ColState& st, int nb_rr, const double* rr_part, int nb_rz,
                          const double* rz_part, int maxit, double rel_trigger, const T* z, T* p, int max_blocks,
                          cudaStream_t s) {
  const int g = grid_for(n, 1, max_blocks);
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
