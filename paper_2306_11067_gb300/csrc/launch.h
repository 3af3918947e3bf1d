// Host-side launchers of the device kernels (explicitly instantiated in
// launch_spmm.cu and launch_level.cu).
#pragma once
#include <vector>

#include "kernels.cuh"
#include "compact.cuh"
#include "separable.cuh"

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
  // FP16 smoother data (T = float, a batch whose columns share lambda): the
  // level's operators below replace ws/we/ga and cf in the V-cycle
  bool h16 = false;
  FineOpH fh{};
  CoarseOpH ch{};
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
// The finest level of the V(1,1) cycle for FP32 vectors (vfine.cuh): down
// = z1 = D^{-1} r, residual and restriction (-> rc); up = z1 + P ec and one
// sweep (-> zout, r.z partials into part when set).  D^{-1} from the stored
// weights (smoother 0: l1-Jacobi, 1: damped Jacobi with omega).  Return
// their block counts.
int launch_vfine_down(const LevelView<float>& L, int B, const float* lam2, int smoother, double omega,
                      const float* r, float* rc, cudaStream_t s);
int launch_vfine_up(const LevelView<float>& L, int B, const float* lam2, int smoother, double omega,
                    const float* r, const float* ec, float* zout, double* part, cudaStream_t s);
template <class T>
void launch_prolong_add(int nvc, int nhc, int B, const T* ec, T* zf, int max_blocks, cudaStream_t s);
template <class T>
void launch_coarse_solve(int nc, int B, const double* kinv, const T* rc, T* ec, cudaStream_t s);

// The small FP16 coarse levels of a V(1,1) cycle and the coarsest solve in
// one single-block kernel per column: levels[0 .. nlev - 2] are the levels
// run there (the first of at most kTailPoints points, FP16 operators), the
// last entry the coarsest level; only levels[0].rhs is read and
// levels[0].z written.  See vtail.cuh.
constexpr int64_t kTailPoints = 1024;  // levels of at most this many points run in the tail kernel
constexpr int64_t kTailCoarsest = 64;  // ... when the coarsest level has at most this many
struct TailLevelIn {
  CoarseOpH op;
  const float* dinv;
  const float* rhs;  // read on the first tail level
  float* z;          // written on the first tail level
};
void launch_vtail(const TailLevelIn* levels, int nlev, const double* kinv, int nc, int B, cudaStream_t s);
bool vtail_fits(int nlev);
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

// ---- separable blur (separable.cu) ----------------------------------------
// One banded 1-D pass in FP64 as built on the host: out(o) = sum_k
// c[k] in(o - H + k), plus the correction rows d of the first nlo and the
// last nhi outputs of a line (empty for a plain correlation).
struct SepPass {
  int H = 0;
  std::vector<double> c;
  int nlo = 0, nhi = 0;
  std::vector<double> d;
};
// the 1-D correlation with taps f (2r + 1 values) or its transpose
SepPass sep_pass_corr(const std::vector<double>& f, bool transpose);
// A^T A of that correlation on a line of len samples (zero boundary)
SepPass sep_pass_ata(const std::vector<double>& f, int len);
// the diagonal of a sep_pass_ata pass (len values)
std::vector<double> sep_diag(const SepPass& p, int len);
// device form of a pass whose correction rows live at d_dev
template <class T>
Band<T> make_band(const SepPass& p, const T* d_dev);
// one pass over every line of an n_v x n_h image and B interleaved columns
// (DIR 0: along i, DIR 1: along j with the epilogue EPI); returns the
// block count (rows of the partial sums when EPI writes any)
template <class T, class TO, int DIR, int EPI>
int launch_band(int nv, int nh, int B, const Band<T>& bd, const T* in, TO* out, const FineOp<T>& fop, const T* P,
                const T* C, const double* lam2, const double* bvec, double* part, int max_blocks, cudaStream_t s);
// opt every k_band instantiation into its shared memory on the current
// device (outside stream capture)
void prepare_band();
// diag(A^T A)_p = dv[i] dh[j]
void launch_sep_diag(int nv, int nh, const double* dv, const double* dh, double* diag, int max_blocks,
                     cudaStream_t s);

}  // namespace lcmg
