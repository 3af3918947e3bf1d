// CSR SpMM launchers: pick the lane split (G column groups x 32/G nnz
// groups, CPG columns per lane) from the batch width.
#include "launch.h"

namespace lcmg {

template <class V, class T, class TO, int G, int CPG, int MODE>
static int run(const SpmmArgs& a0, const V* va, const T* X, TO* Y, const FineOp<T>& fop,
               const T* P, const T* C, const double* lam2, const double* bvec, double* part,
               int max_blocks, cudaStream_t s) {
  SpmmArgs a = a0;
  const int width = G * CPG;
  int64_t blocks = (a.rows + (kBlock / 32) - 1) / (kBlock / 32);
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  dim3 grid((unsigned)blocks, (unsigned)((a.nb + width - 1) / width));
  k_spmm<V, T, TO, G, CPG, MODE><<<grid, kBlock, 0, s>>>(a, va, X, Y, fop, P, C, lam2, bvec, part);
  LCMG_LAUNCHED();
  return (int)blocks;
}

template <class V, class T, class TO, int MODE>
int launch_spmm(const SpmmArgs& a, const V* va, const T* X, TO* Y, const FineOp<T>& fop,
                const T* P, const T* C, const double* lam2, const double* bvec, double* part,
                int max_blocks, cudaStream_t s) {
#define LCMG_RUN(G, CPG) \
  return run<V, T, TO, G, CPG, MODE>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s)
  const int nb = a.nb;
  if (MODE == 0 || MODE == 1) {
    if (nb == 1) LCMG_RUN(1, 1);
    if (nb == 2) LCMG_RUN(2, 1);
    if (nb <= 4) LCMG_RUN(4, 1);
    if (nb <= 8) LCMG_RUN(4, 2);
    if (nb <= 12) LCMG_RUN(4, 3);
    if (nb <= 16) LCMG_RUN(4, 4);
    if (nb <= 20) LCMG_RUN(4, 5);
    if (nb <= 24) LCMG_RUN(4, 6);
    if (nb <= 32) LCMG_RUN(4, 8);
    LCMG_RUN(8, 8);
  } else {
    if (nb == 1) LCMG_RUN(1, 1);
    if (nb <= 8) LCMG_RUN(4, 2);
    if (nb <= 32) LCMG_RUN(4, 8);
    LCMG_RUN(8, 8);
  }
#undef LCMG_RUN
}

#define LCMG_INST(V, T, TO, MODE)                                                             \
  template int launch_spmm<V, T, TO, MODE>(const SpmmArgs&, const V*, const T*, TO*,          \
                                           const FineOp<T>&, const T*, const T*,              \
                                           const double*, const double*, double*, int,        \
                                           cudaStream_t);
// FP32 path
LCMG_INST(float, float, float, 0)
LCMG_INST(float, float, float, 1)
// FP64 path (FP32 or FP64 matrix values)
LCMG_INST(float, double, double, 0)
LCMG_INST(float, double, double, 1)
LCMG_INST(float, double, double, 2)
LCMG_INST(float, double, double, 3)
LCMG_INST(double, double, double, 0)
LCMG_INST(double, double, double, 1)
LCMG_INST(double, double, double, 2)
LCMG_INST(double, double, double, 3)
#undef LCMG_INST

}  // namespace lcmg
