// lcmg_apply_normal_noalloc: the normal-equations operator
// q = (A^T A + lambda^2 L^T D^2 L) p applied without any device allocation.
//
// Some callers cannot allocate device memory where they need this
// operator: code that runs under an external memory manager owning every
// device byte (a framework's caching allocator or a fixed arena), a
// real-time loop that cannot afford an allocation's implicit
// synchronisation and latency, or a thread that must not enter the
// allocator while other threads hold it.  lcmg_apply_normal_dev needs a
// context, and creating a context allocates its workspace.  This entry
// point takes every input and output as a caller-owned device pointer and
// keeps its only intermediate, the vector A p, in a fixed array that is
// part of the library's device image.
#include <cmath>
#include <string>

#include "common.cuh"
#include "lcmg.h"

namespace lcmg {
void set_error_message(const std::string& s);  // capi.cu

namespace noalloc {

// Largest n_cols * m that the intermediate A p may hold: 2^19 doubles
// (4 MiB).  Every GPU that loads the library holds the array until exit.
constexpr int64_t kScratchDoubles = int64_t(1) << 19;
constexpr int kMaxCols = 64;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;

struct Lam2 {  // lambda^2 per column, passed by value (kernel parameter space)
  double v[kMaxCols];
};

// scratch[j * m + r] = (A p_j)[r]; one warp per (row, column)
template <class V>
__global__ void __launch_bounds__(kBlock)
    k_na_forward(int64_t m, int64_t n, int ncols, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                 const V* __restrict__ va, const double* __restrict__ p, double* __restrict__ scratch) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kBlock) >> 5;
  for (int64_t t = warp; t < m * ncols; t += nw) {
    const int j = (int)(t / m);
    const int64_t r = t - (int64_t)j * m;
    const double* pj = p + (int64_t)j * n;
    double s = 0.0;
    for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) s += (double)va[k] * pj[ci[k]];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) scratch[t] = s;
  }
}

// q_j[x] = (A^T scratch_j)[x] + lam2_j (L^T D^2 L p_j)[x]; one warp per
// (pixel, column).  d holds the n_h (n_v - 1) vertical edge weights first
// (edge (i,j)-(i+1,j) at i + j (n_v - 1)), then the (n_h - 1) n_v
// horizontal ones (edge (i,j)-(i,j+1) at n_h (n_v - 1) + i + j n_v).
template <class V>
__global__ void __launch_bounds__(kBlock)
    k_na_normal(int nv, int nh, int64_t m, int ncols, const int64_t* __restrict__ rpT,
                const int32_t* __restrict__ ciT, const V* __restrict__ vaT, const double* __restrict__ d,
                Lam2 lam2, const double* __restrict__ p, const double* __restrict__ scratch,
                double* __restrict__ q) {
  const int lane = threadIdx.x & 31;
  const int64_t n = (int64_t)nv * nh;
  const int64_t nvert = (int64_t)nh * (nv - 1);
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kBlock) >> 5;
  for (int64_t t = warp; t < n * ncols; t += nw) {
    const int col = (int)(t / n);
    const int64_t x = t - (int64_t)col * n;
    const double* sj = scratch + (int64_t)col * m;
    double s = 0.0;
    for (int64_t k = rpT[x] + lane; k < rpT[x + 1]; k += 32) s += (double)vaT[k] * sj[ciT[k]];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      const double* pj = p + (int64_t)col * n;
      const int j = (int)(x / nv), i = (int)(x - (int64_t)j * nv);
      const double px = pj[x];
      double lap = 0.0;
      if (i + 1 < nv) {
        const double w = d[i + (int64_t)j * (nv - 1)];
        lap += w * w * (px - pj[x + 1]);
      }
      if (i > 0) {
        const double w = d[(i - 1) + (int64_t)j * (nv - 1)];
        lap += w * w * (px - pj[x - 1]);
      }
      if (j + 1 < nh) {
        const double w = d[nvert + i + (int64_t)j * nv];
        lap += w * w * (px - pj[x + nv]);
      }
      if (j > 0) {
        const double w = d[nvert + i + (int64_t)(j - 1) * nv];
        lap += w * w * (px - pj[x - nv]);
      }
      q[t] = s + lam2.v[col] * lap;
    }
  }
}

// The device address of g_scratch in the current context, looked up with
// the device current on every call (a cheap query of the loaded module, no
// allocation): a cached address would go stale after cudaDeviceReset or
// under another context of the same device.  In host code the name
// g_scratch denotes a host-side stand-in, never the device array, so only
// this address reaches the kernels.  The first call on a device loads the
// library's device image there if it is not loaded yet, which commits the
// 4 MiB array on that device.
static double* scratch_address() {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess) throw CudaError(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  return static_cast<double*>(ptr);
}

}  // namespace noalloc
}  // namespace lcmg

extern "C" int lcmg_apply_normal_noalloc(int device, void* stream, int32_t n_v, int32_t n_h, int64_t m,
                                         const int64_t* row_ptr, const int32_t* col, const void* val,
                                         const int64_t* row_ptr_t, const int32_t* col_t, const void* val_t,
                                         int32_t val_dtype, const double* d, int32_t n_cols,
                                         const double* lambda, const double* p, double* q) {
  using namespace lcmg;
  int prev = -1;
  int status = LCMG_OK;
  try {
    if (n_v < 2 || n_h < 2 || m < 1 || n_cols < 1 || n_cols > noalloc::kMaxCols || !lambda)
      throw ArgError("bad sizes (need n_v, n_h >= 2, m >= 1, 1 <= n_cols <= 64, lambda != NULL)");
    if (!row_ptr || !col || !val || !row_ptr_t || !col_t || !val_t || !d || !p || !q)
      throw ArgError("null device pointer");
    if (val_dtype != 0 && val_dtype != 1) throw ArgError("val_dtype must be 0 (FP32) or 1 (FP64)");
    if (device < 0 || device >= noalloc::kMaxDevices) throw ArgError("invalid device");
    {  // p is read at neighbouring pixels while q is written: they must not overlap
      const int64_t bytes = (int64_t)n_cols * n_v * n_h * (int64_t)sizeof(double);
      const char* pb = reinterpret_cast<const char*>(p);
      const char* qb = reinterpret_cast<const char*>(q);
      if (pb < qb + bytes && qb < pb + bytes) throw ArgError("p and q overlap");
    }
    if ((int64_t)n_cols * m > noalloc::kScratchDoubles)
      throw ArgError("n_cols * m = " + std::to_string((long long)n_cols * m) +
                     " exceeds the fixed scratch of " + std::to_string((long long)noalloc::kScratchDoubles) +
                     " doubles");
    noalloc::Lam2 l2{};
    for (int j = 0; j < n_cols; ++j) {
      if (!std::isfinite(lambda[j])) throw ArgError("lambda must be finite");
      l2.v[j] = lambda[j] * lambda[j];
    }
    LCMG_CUDA(cudaGetDevice(&prev));
    if (prev != device) LCMG_CUDA(cudaSetDevice(device));
    double* scratch = noalloc::scratch_address();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)n_v * n_h;
    const int bf = (int)std::min<int64_t>((m * n_cols * 32 + kBlock - 1) / kBlock, 4096);
    const int bt = (int)std::min<int64_t>((n * n_cols * 32 + kBlock - 1) / kBlock, 4096);
    // every scratch entry read below is written first: nothing to clear
    if (val_dtype == 0) {
      noalloc::k_na_forward<float><<<bf, kBlock, 0, s>>>(m, n, n_cols, row_ptr, col,
                                                          static_cast<const float*>(val), p, scratch);
      LCMG_LAUNCHED();
      noalloc::k_na_normal<float><<<bt, kBlock, 0, s>>>(n_v, n_h, m, n_cols, row_ptr_t, col_t,
                                                         static_cast<const float*>(val_t), d, l2, p, scratch, q);
      LCMG_LAUNCHED();
    } else {
      noalloc::k_na_forward<double><<<bf, kBlock, 0, s>>>(m, n, n_cols, row_ptr, col,
                                                           static_cast<const double*>(val), p, scratch);
      LCMG_LAUNCHED();
      noalloc::k_na_normal<double><<<bt, kBlock, 0, s>>>(n_v, n_h, m, n_cols, row_ptr_t, col_t,
                                                          static_cast<const double*>(val_t), d, l2, p, scratch, q);
      LCMG_LAUNCHED();
    }
    set_error_message("");
  } catch (const ArgError& e) {
    set_error_message(e.what());
    status = LCMG_ERR_INVALID_ARG;
  } catch (const std::exception& e) {
    set_error_message(e.what());
    status = LCMG_ERR_CUDA;
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return status;
}
