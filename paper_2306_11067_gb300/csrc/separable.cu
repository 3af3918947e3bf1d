// Host side of the separable blur operator: the coefficient sets of the
// banded 1-D passes (built in FP64 from the 1-D PSF factors) and the
// launchers of k_band.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "launch.h"
#include "separable.cuh"

namespace lcmg {

// 1-D correlation A (len x len) with taps f[0..2r]: A[l][l+u] = f[u + r]
// for |u| <= r and 0 <= l + u < len.  The pass for A (transpose false)
// is the correlation itself; for A^T it is the correlation with the
// flipped taps (A^T[i][i-u] = f[u + r]).
SepPass sep_pass_corr(const std::vector<double>& f, bool transpose) {
  const int r = (int)f.size() / 2;
  SepPass p;
  p.H = r;
  p.c.assign(2 * r + 1, 0.0);
  for (int k = 0; k <= 2 * r; ++k) p.c[k] = transpose ? f[2 * r - k] : f[k];
  return p;
}

// T = A^T A of the 1-D correlation above: symmetric, half-bandwidth 2r,
//   T[i][i+k] = sum_{l = 0}^{len-1} f[i - l + r] f[i + k - l + r]
// (terms with |i - l| > r or |i + k - l| > r are zero).  Interior rows hold
// the autocorrelation t_k = sum_u f[u + r] f[u + k + r]; the rows i < r and
// i > len - 1 - r lose the terms with l outside [0, len) and carry the
// difference T[i][i+k] - t_k as their correction row.
SepPass sep_pass_ata(const std::vector<double>& f, int len) {
  const int r = (int)f.size() / 2;
  const int H = 2 * r, taps = 2 * H + 1;
  SepPass p;
  p.H = H;
  p.c.assign(taps, 0.0);
  for (int k = -H; k <= H; ++k) {
    double t = 0.0;
    for (int u = -r; u <= r; ++u)
      if (u + k >= -r && u + k <= r) t += f[u + r] * f[u + k + r];
    p.c[k + H] = t;
  }
  p.nlo = std::min(r, len);
  p.nhi = std::min(r, len - p.nlo);
  auto exact_row = [&](int i, std::vector<double>& row) {
    for (int k = -H; k <= H; ++k) {
      double s = 0.0;
      if (i + k >= 0 && i + k < len)
        for (int l = std::max(0, std::max(i, i + k) - r); l <= std::min(len - 1, std::min(i, i + k) + r); ++l)
          s += f[i - l + r] * f[i + k - l + r];
      // the interior coefficient applies to in(i + k) only where it exists
      const double interior = (i + k >= 0 && i + k < len) ? p.c[k + H] : 0.0;
      row[k + H] = s - interior;
    }
  };
  p.d.assign((size_t)(p.nlo + p.nhi) * taps, 0.0);
  std::vector<double> row(taps);
  for (int i = 0; i < p.nlo; ++i) {
    exact_row(i, row);
    std::copy(row.begin(), row.end(), p.d.begin() + (size_t)i * taps);
  }
  for (int q = 0; q < p.nhi; ++q) {
    exact_row(len - p.nhi + q, row);
    std::copy(row.begin(), row.end(), p.d.begin() + (size_t)(p.nlo + q) * taps);
  }
  return p;
}

// diagonal of T (len values)
std::vector<double> sep_diag(const SepPass& p, int len) {
  const int taps = 2 * p.H + 1;
  std::vector<double> dg(len, p.c[p.H]);
  for (int i = 0; i < p.nlo; ++i) dg[i] += p.d[(size_t)i * taps + p.H];
  for (int q = 0; q < p.nhi; ++q) dg[len - p.nhi + q] += p.d[(size_t)(p.nlo + q) * taps + p.H];
  return dg;
}

template <class T>
Band<T> make_band(const SepPass& p, const T* d_dev) {
  if (p.H < 0 || p.H > kBandMaxH) throw ArgError("band half-width out of range");
  Band<T> b{};
  b.H = p.H;
  b.nch = (2 * p.H + 1 + kBandChunk - 1) / kBandChunk;
  for (int k = 0; k < kBandMaxTaps; ++k) b.c[k] = (k < (int)p.c.size()) ? (T)p.c[k] : (T)0;
  b.nlo = p.d.empty() ? 0 : p.nlo;
  b.nhi = p.d.empty() ? 0 : p.nhi;
  b.d = p.d.empty() ? nullptr : d_dev;
  return b;
}

// blocks of k_band resident at once on the current device
template <class K>
static int band_resident(K kern, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, std::pair<int, size_t>>, int> cache;
  int dev = 0;
  LCMG_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_pair(reinterpret_cast<const void*>(kern), std::make_pair(dev, smem));
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nb = 0, sms = 0;
  LCMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kBandThreads, smem));
  LCMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (nb < 1) throw CudaError("banded pass does not fit on an SM");
  cache[key] = nb * sms;
  return nb * sms;
}

template <class T, class TO, int DIR, int EPI, int TAPS>
static int band_go(int nv, int nh, int B, const Band<T>& bd, const T* in, TO* out, const FineOp<T>& fop, const T* P,
                   const T* C, const double* lam2, const double* bvec, double* part, int max_blocks, cudaStream_t s) {
  auto k = k_band<T, TO, DIR, EPI, TAPS>;
  const size_t smem = band_smem_bytes<T>(bd.nch);
  const int len = DIR == 0 ? nv : nh, lines = DIR == 0 ? nh : nv;
  const int64_t tiles = (int64_t)((len + kBandSeg - 1) / kBandSeg) * ((lines + kBandLines - 1) / kBandLines);
  int64_t blocks = std::min<int64_t>(tiles, band_resident(k, smem));
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, max_blocks));
  klaunch(k, dim3((unsigned)blocks, (unsigned)B), dim3(kBandThreads), smem, s, nv, nh, B, bd, in, out, fop, P, C,
          lam2, bvec, part);
  LCMG_LAUNCHED();
  return (int)blocks;
}

// the A^T A passes of radii 4, 9 and 15 (17, 37 and 61 taps) with their tap
// count compiled in; every other pass with the chunked loop
template <class T, class TO, int DIR, int EPI>
int launch_band(int nv, int nh, int B, const Band<T>& bd, const T* in, TO* out, const FineOp<T>& fop, const T* P,
                const T* C, const double* lam2, const double* bvec, double* part, int max_blocks, cudaStream_t s) {
  constexpr bool kHot = EPI != BAND_RESID2 && !(std::is_same<T, double>::value && DIR == 1 && EPI == BAND_STORE);
  if constexpr (kHot) {
    switch (2 * bd.H + 1) {
      case 17: return band_go<T, TO, DIR, EPI, 17>(nv, nh, B, bd, in, out, fop, P, C, lam2, bvec, part, max_blocks, s);
      case 37: return band_go<T, TO, DIR, EPI, 37>(nv, nh, B, bd, in, out, fop, P, C, lam2, bvec, part, max_blocks, s);
      case 61: return band_go<T, TO, DIR, EPI, 61>(nv, nh, B, bd, in, out, fop, P, C, lam2, bvec, part, max_blocks, s);
      default: break;
    }
  }
  return band_go<T, TO, DIR, EPI, 0>(nv, nh, B, bd, in, out, fop, P, C, lam2, bvec, part, max_blocks, s);
}

template <class T, class TO, int DIR, int EPI>
static void band_optin() {
  const int bytes = (int)band_smem_bytes<T>((2 * kBandMaxH + 1 + kBandChunk - 1) / kBandChunk);
  LCMG_CUDA(cudaFuncSetAttribute(k_band<T, TO, DIR, EPI, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  constexpr bool kHot = EPI != BAND_RESID2 && !(std::is_same<T, double>::value && DIR == 1 && EPI == BAND_STORE);
  if constexpr (kHot) {
    LCMG_CUDA(cudaFuncSetAttribute(k_band<T, TO, DIR, EPI, 17>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    LCMG_CUDA(cudaFuncSetAttribute(k_band<T, TO, DIR, EPI, 37>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    LCMG_CUDA(cudaFuncSetAttribute(k_band<T, TO, DIR, EPI, 61>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  }
}

void prepare_band() {
  band_optin<float, float, 0, BAND_STORE>();
  band_optin<float, float, 1, BAND_NORMAL>();
  band_optin<double, double, 0, BAND_STORE>();
  band_optin<double, double, 1, BAND_STORE>();
  band_optin<double, double, 1, BAND_NORMAL>();
  band_optin<double, double, 1, BAND_RESID2>();
  band_optin<double, double, 1, BAND_TRUERES>();
}

void launch_sep_diag(int nv, int nh, const double* dv, const double* dh, double* diag, int max_blocks,
                     cudaStream_t s) {
  const int64_t n = (int64_t)nv * nh;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, max_blocks));
  klaunch(k_sep_diag, dim3(g), dim3(kBlock), 0, s, nv, nh, dv, dh, diag);
  LCMG_LAUNCHED();
}

template Band<float> make_band<float>(const SepPass&, const float*);
template Band<double> make_band<double>(const SepPass&, const double*);
#define LCMG_BAND_INST(T, TO, DIR, EPI)                                                                          \
  template int launch_band<T, TO, DIR, EPI>(int, int, int, const Band<T>&, const T*, TO*, const FineOp<T>&,    \
                                            const T*, const T*, const double*, const double*, double*, int,     \
                                            cudaStream_t);
LCMG_BAND_INST(float, float, 0, BAND_STORE)
LCMG_BAND_INST(float, float, 1, BAND_NORMAL)
LCMG_BAND_INST(double, double, 0, BAND_STORE)
LCMG_BAND_INST(double, double, 1, BAND_STORE)
LCMG_BAND_INST(double, double, 1, BAND_NORMAL)
LCMG_BAND_INST(double, double, 1, BAND_RESID2)
LCMG_BAND_INST(double, double, 1, BAND_TRUERES)
#undef LCMG_BAND_INST

}  // namespace lcmg
