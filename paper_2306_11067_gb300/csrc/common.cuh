// Shared definitions of the lcmg CUDA library (sm_103a).
//
// Batched vectors are stored interleaved: element (point p, column j) of an
// n x B batch lives at p * B + j, so the B systems (one per lambda and
// right-hand side) that share an operator read each operator coefficient
// once and their values for one point from one contiguous run of memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

namespace lcmg {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct ArgError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct MemError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define LCMG_CUDA(call)                                                             \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::lcmg::CudaError(std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
// Kernels launched by this thread (every launch site is followed by
// LCMG_LAUNCHED(); graph replays add the kernels of the captured block).
inline int64_t& launch_counter() {
  static thread_local int64_t count = 0;
  return count;
}
#define LCMG_LAUNCHED()                  \
  do {                                   \
    ++::lcmg::launch_counter();          \
    LCMG_CUDA(cudaGetLastError());       \
  } while (0)

// Asynchronous global -> shared copies of one element (cp.async, 4 or 8
// bytes), zero-filled when `valid` is false (source size 0; the source
// address is then `fallback`, an address inside the array, and no byte is
// read).  A thread issues all of its copies of a tile before it waits, so a
// block keeps its whole tile's loads in flight instead of one per thread.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* src, const T* fallback, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  const T* g = valid ? src : fallback;
  const int n = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(g), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(g), "r"(n) : "memory");
}
// 16 bytes (both addresses 16-byte aligned), zero-filled when !valid
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* src, const void* fallback, bool valid) {
  const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  const void* g = valid ? src : fallback;
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(g), "r"(n) : "memory");
}
// wait for every cp.async this thread issued (a __syncthreads must follow
// before other threads read the copied data)
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// close the group of copies issued so far; wait until at most N groups of
// this thread are still in flight
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kBlock = 256;      // threads per block of the point x column kernels
constexpr int kMaxB = 256;       // widest batch one launch handles
constexpr int kStencil = 25;     // coarse-level stencils are 5 x 5

// per-column solve state codes (device side)
enum : int { ST_CONVERGED = 0, ST_MAXIT = 1, ST_BREAKDOWN = 2, ST_NONFINITE = 3, ST_RUNNING = 9 };

// ---------------------------------------------------------------------------
// Point x column thread mapping: a block of kBlock threads covers
// pts = kBlock / B points for all B columns; thread t handles column
// t % B of point (block's first point) + t / B.
// ---------------------------------------------------------------------------
struct ColMap {
  int B, pts, k, col;
  bool ok;
  __device__ __forceinline__ explicit ColMap(int B_) : B(B_) {
    pts = kBlock / B;
    k = threadIdx.x / B;
    col = threadIdx.x - k * B;
    ok = k < pts;
  }
  __device__ __forceinline__ int64_t first() const { return (int64_t)blockIdx.x * pts + k; }
  __device__ __forceinline__ int64_t stride() const { return (int64_t)gridDim.x * pts; }
};

// Deterministic per-column block reduction: sums v over the pts points of
// the block for every column and writes out[col] (one value per column).
// All threads of the block must call it.
__device__ __forceinline__ void block_col_sum(double v, const ColMap& cm, double* smem,
                                              double* out) {
  smem[threadIdx.x] = cm.ok ? v : 0.0;
  int p2 = 1;
  while (p2 < cm.pts) p2 <<= 1;
  for (int s = p2 >> 1; s > 0; s >>= 1) {
    __syncthreads();
    if (cm.ok && cm.k < s && cm.k + s < cm.pts) smem[threadIdx.x] += smem[threadIdx.x + s * cm.B];
  }
  __syncthreads();
  if (cm.ok && cm.k == 0) out[cm.col] = smem[cm.col];
  __syncthreads();
}

__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(double v) { return v; }

template <class T>
__device__ __forceinline__ T from_d(double v);
template <>
__device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ double from_d<double>(double v) { return v; }

// Launch kern on stream s (every launch of the library goes through here).
template <typename... KArgs, typename... Args>
inline void klaunch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  LCMG_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}

inline int grid_for(int64_t points, int B, int max_blocks) {
  int pts = kBlock / B;
  int64_t g = (points + pts - 1) / pts;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace lcmg
