// CSR SpMM launchers: pick the lane split (G column groups x 32/G nnz
// groups, CPG columns per lane) from the batch width.
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "launch.h"

namespace lcmg {

// Blocks of a kernel that are resident at once on the current device (the
// grid of one full wave): a grid-stride kernel launched with more blocks
// than this runs a second, partial wave.
template <class K>
static int resident_grid(K kern, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  LCMG_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_pair(reinterpret_cast<const void*>(kern), dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nb = 0, sms = 0;
  LCMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem));
  LCMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (nb < 1) nb = 1;
  cache[key] = nb * sms;
  return nb * sms;
}

// One column: k_spmv1 with U nonzeros per lane and LPR lanes per row;
// 16-bit column offsets (C16) in the 8-lane layout when present.
template <class V, class T, class TO, int MODE, int U, int LPR, bool C16, int MINB>
static int run1c(const SpmmArgs& a, const V* va, const T* X, TO* Y, const FineOp<T>& fop, const T* P,
                 const T* C, const double* lam2, const double* bvec, double* part, int max_blocks,
                 cudaStream_t s) {
  auto k = k_spmv1<V, T, TO, MODE, U, LPR, true, C16, MINB>;
  int64_t blocks = resident_grid(k, kBlock, 0);
  const int64_t need = (a.rows * LPR + kBlock - 1) / kBlock;
  if (blocks > need) blocks = need;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  klaunch(k, dim3((unsigned)blocks), dim3(kBlock), 0, s, a, va, X, Y, fop, P, C, lam2, bvec, part);
  LCMG_LAUNCHED();
  return (int)blocks;
}

template <class V, class T, class TO, int MODE, int U, int LPR, int MINB = spmv1_minb<T, LPR>()>
static int run1v(const SpmmArgs& a, const V* va, const T* X, TO* Y, const FineOp<T>& fop, const T* P,
                 const T* C, const double* lam2, const double* bvec, double* part, int max_blocks,
                 cudaStream_t s) {
  // 16-bit columns in the 8-lane layout (the transposed pass): measured on
  // GB300 (ct256) it gains (38.2 -> 35.3 us per pass), while y = A p in the
  // 32-lane layout under a 32-register cap loses (31.1 -> 38.3 us) and keeps
  // int32 columns
  if constexpr ((MODE == 0 || MODE == 1) && LPR == 8) {
    if (a.c16 != nullptr)
      return run1c<V, T, TO, MODE, U, LPR, true, MINB>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
  }
  return run1c<V, T, TO, MODE, U, LPR, false, MINB>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
}

// The pass's configuration: a.variant, or by default (measured on GB300,
// 256^2 CT) 32 lanes x 4 for y = A p and 8 lanes x 8 for the transposed
// pass, whose fine-level epilogue runs on one lane per row (with FP32
// vectors compiled for 5 resident blocks per SM).
template <class V, class T, class TO, int MODE>
static int run1(const SpmmArgs& a, const V* va, const T* X, TO* Y, const FineOp<T>& fop, const T* P,
                const T* C, const double* lam2, const double* bvec, double* part, int max_blocks,
                cudaStream_t s) {
  constexpr bool kT = (MODE == 1 || MODE == 3);
  // transposed pass with FP32 vectors: 8 x 8 bounded to 5 blocks per SM
  // (48 registers; 32.8 vs 35.7-36.2 us per pass on GB300, same sums)
  const int v = a.variant != 0 ? a.variant : (kT ? (std::is_same<T, float>::value ? 4 : 3) : 1);
  if (v == 2) return run1v<V, T, TO, MODE, 8, 16>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
  if constexpr (std::is_same<T, float>::value) {  // register-bounded forms of the 8-lane layout
    if (v == 4) return run1v<V, T, TO, MODE, 8, 8, 5>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
    if (v == 5) return run1v<V, T, TO, MODE, 8, 8, 6>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
    if (v == 6) return run1v<V, T, TO, MODE, 4, 8, 8>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
  }
  if (v >= 3) return run1v<V, T, TO, MODE, 8, 8>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
  return run1v<V, T, TO, MODE, 4, 32>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
}

template <class V, class T, class TO, int G, int CPG, int MODE>
static int run(const SpmmArgs& a0, const V* va, const T* X, TO* Y, const FineOp<T>& fop,
               const T* P, const T* C, const double* lam2, const double* bvec, double* part,
               int max_blocks, cudaStream_t s) {
  SpmmArgs a = a0;
  const int width = G * CPG;
  if (G == 1 && CPG == 1) return run1<V, T, TO, MODE>(a, va, X, Y, fop, P, C, lam2, bvec, part, max_blocks, s);
  auto k = k_spmm<V, T, TO, G, CPG, MODE>;
  int64_t blocks = (a.rows + (kBlock / 32) - 1) / (kBlock / 32);
  const int64_t wave = resident_grid(k, kBlock, 0);
  if (blocks > wave) blocks = wave;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  dim3 grid((unsigned)blocks, (unsigned)((a.nb + width - 1) / width));
  klaunch(k, dim3(grid), dim3(kBlock), 0, s, a, va, X, Y, fop, P, C, lam2, bvec, part);
  LCMG_LAUNCHED();
  return (int)blocks;
}

// Lane split (G column groups, CPG columns per lane) for a batch of nb
// columns: f(integral_constant<G>, integral_constant<CPG>).
template <int MODE, class F>
static int dispatch_split(int nb, F&& f) {
  using std::integral_constant;
  if (MODE == 0 || MODE == 1) {
    if (nb == 1) return f(integral_constant<int, 1>{}, integral_constant<int, 1>{});
    if (nb == 2) return f(integral_constant<int, 2>{}, integral_constant<int, 1>{});
    if (nb <= 4) return f(integral_constant<int, 4>{}, integral_constant<int, 1>{});
    if (nb <= 8) return f(integral_constant<int, 4>{}, integral_constant<int, 2>{});
    if (nb <= 12) return f(integral_constant<int, 4>{}, integral_constant<int, 3>{});
    if (nb <= 16) return f(integral_constant<int, 4>{}, integral_constant<int, 4>{});
    if (nb <= 20) return f(integral_constant<int, 4>{}, integral_constant<int, 5>{});
    if (nb <= 24) return f(integral_constant<int, 4>{}, integral_constant<int, 6>{});
    if (nb <= 32) return f(integral_constant<int, 4>{}, integral_constant<int, 8>{});
    return f(integral_constant<int, 8>{}, integral_constant<int, 8>{});
  }
  if (nb == 1) return f(integral_constant<int, 1>{}, integral_constant<int, 1>{});
  if (nb <= 8) return f(integral_constant<int, 4>{}, integral_constant<int, 2>{});
  if (nb <= 32) return f(integral_constant<int, 4>{}, integral_constant<int, 8>{});
  return f(integral_constant<int, 8>{}, integral_constant<int, 8>{});
}

template <class V, class T, class TO, int MODE>
int launch_spmm(const SpmmArgs& a, const V* va, const T* X, TO* Y, const FineOp<T>& fop,
                const T* P, const T* C, const double* lam2, const double* bvec, double* part,
                int max_blocks, cudaStream_t s) {
  return dispatch_split<MODE>(a.nb, [&](auto g, auto cpg) {
    return run<V, T, TO, decltype(g)::value, decltype(cpg)::value, MODE>(a, va, X, Y, fop, P, C, lam2, bvec,
                                                                         part, max_blocks, s);
  });
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
