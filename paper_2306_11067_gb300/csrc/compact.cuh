// FP16 storage of the V-cycle's smoother data (mixed precision, a batch
// whose columns share one lambda: the paper's chain and its right-hand-side
// batches).
//
// A V-cycle only has to be a fixed symmetric positive definite operator for
// PCG; its level operators need not be exact.  On the one-column chain the
// smoother data is most of what the cycle reads (a coarse point's stencil
// is 25 + 25 coefficients against one vector entry), so it is stored in
// FP16, each array scaled by a power of two that puts its largest value
// just below 2^13:
//
//  * finest level: the squared edge weights w_s, w_e and diag(A^T A), FP16
//    (lambda-independent, rebuilt with the weights); the cycle forms
//    lam^2 L^T W^ L + diag(ga^) from them, so the level operator keeps the
//    structure of the exact one (a weighted graph Laplacian plus a positive
//    diagonal) with every weight rounded to 11 significant bits;
//  * coarse level k: per lambda, the 24 off-diagonal coefficients of
//    K_k(lam) = lam^2 G_L^k + G_A^k, FP16 (48 bytes per point against 256
//    for the FP32 rows of both parts), and the row sums s = G_A^k 1 in FP32
//    (lambda-independent: the rows of G_L^k sum to zero); the diagonal is
//    s_p minus the sum of the stored off-diagonals, so K^ 1 = G_A 1 exactly
//    and the rounding perturbs K by a zero-row-sum (Laplacian-like) term of
//    relative size 2^-11 that keeps it positive definite.
//
// The coarsest level keeps its exact FP64 factorisation.  Tested against
// the oracle's model of the same storage (oracle.multigrid, storage="fp16").
#pragma once
#include <cuda_fp16.h>

#include <cmath>

#include "kernels.cuh"

namespace lcmg {

constexpr int kCompactOff = 24;     // stored coefficients per coarse point
constexpr double kHalfTarget = 8192.0;  // scaled maxima lie in (4096, 8192]

// power of two putting max (> 0) in (kHalfTarget / 2, kHalfTarget]
inline double half_scale(double max) {
  if (!(max > 0.0)) return 1.0;
  return std::ldexp(1.0, (int)std::floor(std::log2(kHalfTarget / max)));
}

// finest level in FP16: the operator of FineOp with rounded weights
struct FineOpH {
  int nv, nh;
  const __half* __restrict__ ws;  // w_s 2^e_w
  const __half* __restrict__ we;  // w_e 2^e_w
  const __half* __restrict__ ga;  // diag(A^T A) 2^e_g
  float sw, sg;                   // 2^-e_w, 2^-e_g
  static constexpr int kRadius = 1;

  __device__ __forceinline__ float ws_(int64_t p) const { return __half2float(ws[p]) * sw; }
  __device__ __forceinline__ float we_(int64_t p) const { return __half2float(we[p]) * sw; }
  __device__ __forceinline__ float ga_(int64_t p) const { return __half2float(ga[p]) * sg; }

  template <class F>
  __device__ __forceinline__ float lap(int64_t p, int i, int j, F v) const {
    const float zp = v(p);
    float acc = 0;
    if (i + 1 < nv) acc += ws_(p) * (zp - v(p + 1));
    if (i > 0) acc += ws_(p - 1) * (zp - v(p - 1));
    if (j + 1 < nh) acc += we_(p) * (zp - v(p + nv));
    if (j > 0) acc += we_(p - nv) * (zp - v(p - nv));
    return acc;
  }
  template <class F>
  __device__ __forceinline__ float apply(int64_t p, int i, int j, float lam2, F v) const {
    return lam2 * lap(p, i, j, v) + ga_(p) * v(p);
  }
  template <class F>
  __device__ __forceinline__ float apply_off(int64_t p, int i, int j, float lam2, F v) const {
    const float zp = v(0, 0);
    float acc = 0;
    if (i + 1 < nv) acc += ws_(p) * (zp - v(1, 0));
    if (i > 0) acc += ws_(p - 1) * (zp - v(-1, 0));
    if (j + 1 < nh) acc += we_(p) * (zp - v(0, 1));
    if (j > 0) acc += we_(p - nv) * (zp - v(0, -1));
    return lam2 * acc + ga_(p) * zp;
  }
  __device__ __forceinline__ double diagL(int64_t p, int i, int j) const {
    double s = 0;
    if (i + 1 < nv) s += (double)ws_(p);
    if (i > 0) s += (double)ws_(p - 1);
    if (j + 1 < nh) s += (double)we_(p);
    if (j > 0) s += (double)we_(p - nv);
    return s;
  }
  __device__ __forceinline__ double l1(int64_t p, int i, int j, double lam2) const {
    return 2.0 * lam2 * diagL(p, i, j) + (double)ga_(p);
  }
  __device__ __forceinline__ double center(int64_t p, int i, int j, double lam2) const {
    return lam2 * diagL(p, i, j) + (double)ga_(p);
  }
};

// coarse level in FP16: row p holds the off-diagonal coefficients of
// K(lam) for the offsets o = (di+2) + 5 (dj+2) in increasing o, o = 12 left
// out, scaled by 2^e; the diagonal is s[p] minus their sum
struct CoarseOpH {
  int nv, nh;
  int64_t n;
  const uint4* __restrict__ rows;  // 3 x 16 bytes per point
  const float* __restrict__ s;     // row sums of G_A
  float sc;                        // 2^-e
  static constexpr int kRadius = 2;

  // k[o] of K(lam) for o < 25 (lam2 is already in the stored rows)
  __device__ __forceinline__ void coefs(int64_t p, float, float (&k)[28]) const {
    decode(rows[3 * p], rows[3 * p + 1], rows[3 * p + 2], s[p], k);
  }
  // the same from a row's three 16-byte words and its row sum
  __device__ __forceinline__ void decode(const uint4 q0, const uint4 q1, const uint4 q2, const float sp,
                                        float (&k)[28]) const {
    const uint32_t w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
    float off[kCompactOff];
#pragma unroll
    for (int h = 0; h < 12; ++h) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[h]));
      off[2 * h] = f.x * sc;
      off[2 * h + 1] = f.y * sc;
    }
    float sum = 0;
#pragma unroll
    for (int o = 0; o < kCompactOff; ++o) sum += off[o];
#pragma unroll
    for (int o = 0; o < 12; ++o) k[o] = off[o];
    k[12] = sp - sum;
#pragma unroll
    for (int o = 13; o < 25; ++o) k[o] = off[o - 1];
    k[25] = k[26] = k[27] = 0;
  }
  // (K v)_p from the point's three row words and row sum, every one of the
  // 25 terms taken (the caller's v is zero outside the grid, so the terms
  // apply_k leaves out add nothing).  The products are formed with the
  // stored FP16 values and the sum scaled by sc at the end: sc and its
  // inverse are powers of two, so every product and partial sum is the one
  // apply_k forms, times 2^e exactly, and the result is the same float.
  template <class F>
  __device__ __forceinline__ float apply_rows(const uint4 q0, const uint4 q1, const uint4 q2, const float sp,
                                              float inv_sc, F v) const {
    const uint32_t w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
    float off[kCompactOff];
#pragma unroll
    for (int h = 0; h < 12; ++h) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[h]));
      off[2 * h] = f.x;
      off[2 * h + 1] = f.y;
    }
    float sum = 0;
#pragma unroll
    for (int o = 0; o < kCompactOff; ++o) sum += off[o];
    const float center = sp * inv_sc - sum;
    float acc = 0;
#pragma unroll
    for (int o = 0; o < 25; ++o) {
      const int dj = o / 5 - 2, di = o % 5 - 2;
      const float k = o < 12 ? off[o] : (o == 12 ? center : off[o - 1]);
      acc += k * v(di, dj);
    }
    return acc * sc;
  }
  template <class F>
  __device__ __forceinline__ float apply_k(const float (&k)[28], int i, int j, F v) const {
    float acc = 0;
    if (i >= 2 && i + 2 < nv && j >= 2 && j + 2 < nh) {
#pragma unroll
      for (int dj = -2; dj <= 2; ++dj)
#pragma unroll
        for (int di = -2; di <= 2; ++di) acc += k[(di + 2) + 5 * (dj + 2)] * v(di, dj);
      return acc;
    }
#pragma unroll
    for (int dj = -2; dj <= 2; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= nh) continue;
#pragma unroll
      for (int di = -2; di <= 2; ++di) {
        const int ii = i + di;
        if (ii < 0 || ii >= nv) continue;
        acc += k[(di + 2) + 5 * (dj + 2)] * v(di, dj);
      }
    }
    return acc;
  }
  template <class F>
  __device__ __forceinline__ float apply_off(int64_t p, int i, int j, float lam2, F v) const {
    float k[28];
    coefs(p, lam2, k);
    return apply_k(k, i, j, v);
  }
  template <class F>
  __device__ __forceinline__ float apply(int64_t p, int i, int j, float lam2, F v) const {
    auto vo = [&](int di, int dj) { return v((int64_t)(i + di) + (int64_t)(j + dj) * nv); };
    return apply_off(p, i, j, lam2, vo);
  }
  __device__ __forceinline__ double l1(int64_t p, int, int, double) const {
    float k[28];
    coefs(p, 0.f, k);
    double s1 = 0;
    for (int o = 0; o < kStencil; ++o) s1 += fabs((double)k[o]);
    return s1;
  }
  __device__ __forceinline__ double center(int64_t p, int, int, double) const {
    float k[28];
    coefs(p, 0.f, k);
    return (double)k[12];
  }
};

// dst = fp16(src * scale), rounded to nearest from FP64
static __global__ void k_half_scaled(int64_t n, const double* __restrict__ src, double scale,
                                     __half* __restrict__ dst) {
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock)
    dst[p] = __double2half(src[p] * scale);
}

// s[p] = sum_o g[o][p] (25 x n SoA, o in increasing order), in FP32
static __global__ void k_rowsum25(int64_t n, const double* __restrict__ g, float* __restrict__ s) {
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    double t = 0.0;
    for (int o = 0; o < kStencil; ++o) t += g[(int64_t)o * n + p];
    s[p] = (float)t;
  }
}

// *mx = max |v| over v (n values, or the 24 off-diagonal rows of a 25 x n
// SoA stencil when stencil25); non-negative doubles order like their bits
static __global__ void k_maxabs(int64_t n, const double* __restrict__ v, int stencil25,
                                unsigned long long* __restrict__ mx) {
  double m = 0.0;
  const int rows = stencil25 ? kStencil : 1;
  for (int o = 0; o < rows; ++o) {
    if (stencil25 && o == 12) continue;
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock)
      m = fmax(m, fabs(v[(int64_t)o * n + p]));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

// the coarse rows of K(lam) = lam2 G_L + G_A (off-diagonals, FP16, x scale)
static __global__ void k_compact_rows(int64_t n, const double* __restrict__ gl, const double* __restrict__ ga,
                                      double lam2, double scale, __half* __restrict__ rows) {
  for (int64_t t = (int64_t)blockIdx.x * kBlock + threadIdx.x; t < n * kCompactOff;
       t += (int64_t)gridDim.x * kBlock) {
    const int64_t p = t / kCompactOff;
    const int h = (int)(t - p * kCompactOff);
    const int o = h < 12 ? h : h + 1;
    const double k = lam2 * gl[(int64_t)o * n + p] + ga[(int64_t)o * n + p];
    rows[t] = __double2half(k * scale);
  }
}

}  // namespace lcmg
