// Host-side launchers of the device kernels (explicitly instantiated in
// launch_spmm.cu and launch_level.cu).
#pragma once
#include "kernels.cuh"

namespace lcmg {

// Level operator view for one precision.
template <class T>
struct LevelView {
  int nv = 0, nh = 0;
  int64_t n = 0;
  bool fine = true;
  const T* ws = nullptr;  // fine level: squared edge weights
  const T* we = nullptr;
  const T* ga = nullptr;  // fine: diag(A^T A)
  const T* cf = nullptr;  // coarse: per-point coefficient rows
  FineOp<T> fine_op() const { return FineOp<T>{nv, nh, ws, we, ga}; }
  CoarseOp<T> coarse_op() const { return CoarseOp<T>{nv, nh, n, cf}; }
};

// Y = A X / Q = A^T Y + lam2 L^T W L P (+dot) / rho partials / true residual.
// Returns the number of blocks (rows of the partial-sum array).
template <class V, class T, class TO, int MODE>
int launch_spmm(const SpmmArgs& a, const V* va, const T* X, TO* Y, const FineOp<T>& fop,
                const T* P, const T* C, const double* lam2, const double* bvec, double* part,
                int max_blocks, cudaStream_t s);

template <class T>
void launch_dinv(const LevelView<T>& L, int B, const double* lam2, int smoother, double omega,
                 T* dinv, int max_blocks, cudaStream_t s);
template <class T>
void launch_smooth_zero(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r,
                        T* z, int two, int max_blocks, cudaStream_t s);
// returns the number of partial blocks when part != nullptr
template <class T>
int launch_smooth(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r,
                  const T* zin, T* zout, const int* active, double* part, int max_blocks,
                  cudaStream_t s);
template <class T>
void launch_residual(const LevelView<T>& L, int B, const T* lam2, const T* r, const T* z, T* res,
                     int max_blocks, cudaStream_t s);
template <class T>
void launch_restrict(int nvc, int nhc, int B, const T* rf, T* rc, int max_blocks, cudaStream_t s);
// Level k of the V-cycle in two kernels (nu = 1 or 2 sweeps): down = pre-
// smoothing from zero, residual and restriction (z -> zpre, R res -> rc);
// up = zpre + P ec followed by nu sweeps (-> zout; r.z partials into part
// when part is set).  Both return their block count (tiles).
template <class T>
int launch_vdown(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r, T* zpre, T* rc,
                 int nu, cudaStream_t s);
template <class T>
int launch_vup(const LevelView<T>& L, int B, const T* lam2, const T* dinv, const T* r, const T* ec,
               const T* zpre, T* zout, double* part, int nu, cudaStream_t s);
template <class T>
void launch_prolong_add(int nvc, int nhc, int B, const T* ec, T* zf, int max_blocks, cudaStream_t s);
template <class T>
void launch_coarse_solve(int nc, int B, const double* kinv, const T* rc, T* ec, cudaStream_t s);
void launch_dense_setup(const LevelView<double>& L, int B, const double* lam2, double* M,
                        double* W, double* K, int* info, int max_blocks, cudaStream_t s);
void launch_galerkin(const RapIn& in, int nvc, int nhc, double* out, int max_blocks, cudaStream_t s);

template <class T, class TX>
int launch_update_xr(int64_t n, int B, const ColState& st, const T* p, const T* q, TX* x, T* r,
                     double* part, int max_blocks, cudaStream_t s);
// one column: alpha from the p.q partials inside the update (no scalar kernel)
template <class T, class TX>
int launch_update_xr_alpha(int64_t n, const ColState& st, int nb_pq, const double* pq_part, const T* p,
                           const T* q, TX* x, T* r, double* part, int max_blocks, cudaStream_t s);
template <class T>
void launch_update_p(int64_t n, int B, const ColState& st, const T* z, T* p, int max_blocks,
                     cudaStream_t s);
// one column, keep = 0: beta from the r.r and r.z partials inside the p update
template <class T>
void launch_update_p_beta(int64_t n, const ColState& st, int nb_rr, const double* rr_part, int nb_rz,
                          const double* rz_part, int maxit, double rel_trigger, const T* z, T* p, int max_blocks,
                          cudaStream_t s);
template <class T>
void launch_copy_cols(int64_t n, int B, const int* flag, const T* src, T* dst, int max_blocks,
                      cudaStream_t s);

}  // namespace lcmg
