// PMIS C/F split on the device: the parallel replacement of the greedy
// first and second passes of Sec. 3.1 (rules in rs_amg.h).  The strength
// sets S and S^T come from the host (amg::strength); every round is three
// kernels over the points, and no decision depends on the order in which
// threads run, so the split is deterministic.
#include <algorithm>

#include "common.cuh"
#include "rs_amg.h"

namespace lcmg {
namespace amg {

constexpr int8_t kU = -1;

// uniform in [0, 1) of output i of the SplitMix64 stream seeded with seed
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, int64_t i) {
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

static __global__ void k_pmis_init(int64_t n, const int64_t* __restrict__ srp, const int64_t* __restrict__ trp,
                                   uint64_t seed, double* __restrict__ w, int8_t* __restrict__ st) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t deps = trp[i + 1] - trp[i];
    w[i] = (double)deps + splitmix_uniform(seed, i);
    st[i] = (deps == 0 && srp[i + 1] == srp[i]) ? kF : kU;
  }
}

// newc[i] = 1: unsorted i whose (measure, index) exceeds that of every
// unsorted point it is strongly connected to, in either direction
static __global__ void k_pmis_select(int64_t n, const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
                                     const int64_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                     const double* __restrict__ w, const int8_t* __restrict__ st,
                                     int8_t* __restrict__ newc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int8_t pick = 0;
    if (st[i] == kU) {
      const double wi = w[i];
      bool best = true;
      for (int64_t k = srp[i]; k < srp[i + 1] && best; ++k) {
        const int32_t j = sci[k];
        if (st[j] == kU && !(wi > w[j] || (wi == w[j] && i > j))) best = false;
      }
      for (int64_t k = trp[i]; k < trp[i + 1] && best; ++k) {
        const int32_t j = tci[k];
        if (st[j] == kU && !(wi > w[j] || (wi == w[j] && i > j))) best = false;
      }
      pick = best ? 1 : 0;
    }
    newc[i] = pick;
  }
}

static __global__ void k_pmis_apply(int64_t n, const int8_t* __restrict__ newc, int8_t* __restrict__ st) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (newc[i]) st[i] = kC;
}

// unsorted points with a strong connection to a C point become F (a write
// turns U into F only, and reads test for C only, so concurrent threads
// agree); the others are counted
static __global__ void k_pmis_f(int64_t n, const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
                                int8_t* __restrict__ st, int* __restrict__ left) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (st[i] != kU) continue;
    bool f = false;
    for (int64_t k = srp[i]; k < srp[i + 1] && !f; ++k) f = st[sci[k]] == kC;
    if (f) st[i] = kF;
    else atomicAdd(left, 1);
  }
}

namespace {
struct Dev {
  void* p = nullptr;
  explicit Dev(size_t bytes) {
    if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) {
      cudaGetLastError();
      throw MemError("device allocation for the PMIS split failed");
    }
  }
  ~Dev() {
    if (p) cudaFree(p);
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};
}  // namespace

std::vector<int8_t> pmis_split(const Strength& S, int64_t n, uint64_t seed, cudaStream_t s) {
  // S^T in increasing row order
  Strength T;
  T.rp.assign(n + 1, 0);
  for (int32_t j : S.ci) T.rp[j + 1]++;
  for (int64_t i = 0; i < n; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(S.ci.size());
  {
    std::vector<int64_t> pos(T.rp.begin(), T.rp.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k) T.ci[pos[S.ci[k]]++] = (int32_t)i;
  }
  const size_t nz = S.ci.size();
  Dev srp(sizeof(int64_t) * (n + 1)), sci(sizeof(int32_t) * nz), trp(sizeof(int64_t) * (n + 1)),
      tci(sizeof(int32_t) * nz), w(sizeof(double) * n), st(n), newc(n), left(sizeof(int));
  LCMG_CUDA(cudaMemcpyAsync(srp.p, S.rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  LCMG_CUDA(cudaMemcpyAsync(sci.p, S.ci.data(), sizeof(int32_t) * nz, cudaMemcpyHostToDevice, s));
  LCMG_CUDA(cudaMemcpyAsync(trp.p, T.rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  LCMG_CUDA(cudaMemcpyAsync(tci.p, T.ci.data(), sizeof(int32_t) * nz, cudaMemcpyHostToDevice, s));
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 4096);
  klaunch(k_pmis_init, dim3(blocks), dim3(threads), 0, s, n, (const int64_t*)srp.as<int64_t>(),
          (const int64_t*)trp.as<int64_t>(), seed, w.as<double>(), st.as<int8_t>());
  LCMG_LAUNCHED();
  // every round makes the unsorted point of largest (measure, index) C, so
  // at most n rounds
  for (int64_t round = 0;; ++round) {
    if (round > n) throw CudaError("PMIS split did not finish within n rounds");
    klaunch(k_pmis_select, dim3(blocks), dim3(threads), 0, s, n, (const int64_t*)srp.as<int64_t>(),
            (const int32_t*)sci.as<int32_t>(), (const int64_t*)trp.as<int64_t>(), (const int32_t*)tci.as<int32_t>(),
            (const double*)w.as<double>(), (const int8_t*)st.as<int8_t>(), newc.as<int8_t>());
    LCMG_LAUNCHED();
    klaunch(k_pmis_apply, dim3(blocks), dim3(threads), 0, s, n, (const int8_t*)newc.as<int8_t>(), st.as<int8_t>());
    LCMG_LAUNCHED();
    LCMG_CUDA(cudaMemsetAsync(left.p, 0, sizeof(int), s));
    klaunch(k_pmis_f, dim3(blocks), dim3(threads), 0, s, n, (const int64_t*)srp.as<int64_t>(),
            (const int32_t*)sci.as<int32_t>(), st.as<int8_t>(), left.as<int>());
    LCMG_LAUNCHED();
    int h = 0;
    LCMG_CUDA(cudaMemcpyAsync(&h, left.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    LCMG_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
  }
  std::vector<int8_t> cf(n);
  LCMG_CUDA(cudaMemcpyAsync(cf.data(), st.p, n, cudaMemcpyDeviceToHost, s));
  LCMG_CUDA(cudaStreamSynchronize(s));
  return cf;
}

}  // namespace amg
}  // namespace lcmg
