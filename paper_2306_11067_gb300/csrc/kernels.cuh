// Device kernels of the multigrid-preconditioned CG solver.
//
// Operators (paper sections in brackets):
//   * K(lam) = A^T A + lam^2 L^T D^2 L, applied in two stages: y = A p (CSR
//     SpMM), then q = A^T y + lam^2 L^T W L p with W = D^2 (transposed CSR,
//     no atomics) with the dot p^T q fused  [Sec. 3.2, eq. (normal)].
//   * The V-cycle operator K_pre(lam) = lam^2 G_L + G_A with G_L^0 = L^T W L
//     (5-point, variable coefficient) and G_A^0 = diag(A^T A); coarse levels
//     are Galerkin products P^T G P with cell-centred bilinear P, which are
//     5 x 5 (25-point) stencils  [Sec. 3.1, Algorithm 1].
#pragma once
#include "common.cuh"

namespace lcmg {

// ---------------------------------------------------------------------------
// 1-D cell-centred linear interpolation weight P(a, I) from coarse cell I
// (of nc) to fine cell a (of 2 nc): 3/4 from the parent, 1/4 from the
// nearest other coarse cell; a missing neighbour's weight goes to the parent.
// ---------------------------------------------------------------------------
// (In the precision of the kernel that uses it: the weights 1, 3/4, 1/4
// are exact in any format, and an FP32 kernel then needs no FP64 work.)
template <class T = double>
__device__ __forceinline__ T pw1(int a, int I, int nc) {
  const int d = a - 2 * I;
  if (d == 0) return I == 0 ? T(1) : T(0.75);
  if (d == 1) return I == nc - 1 ? T(1) : T(0.75);
  if (d == -1 || d == 2) return T(0.25);
  return T(0);
}

// Compensated dot product in the working precision (Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005, Algorithm Dot2): each product is
// split exactly into p + e with one FMA, the running sum is kept exact to
// rounding as s + c with TwoSum, so the result is as accurate as a dot
// product in twice the working precision.  The mixed path's FP32 kernels
// accumulate their dot products this way and convert s + c to FP64 once per
// thread: on this GPU the FP64 pipe runs at a small fraction of the FP32 one.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);  // a b = p + e exactly
    const float t = s + p;
    const float z = t - s;
    c += (s - (t - z)) + (p - z) + e;  // TwoSum error of s + p, plus e
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// A thread's dot-product accumulator: FP64 for FP64 vectors, Dot2 for FP32
template <class T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s += a * b; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> : Dot2 {};

// ---------------------------------------------------------------------------
// Level operators
// ---------------------------------------------------------------------------
// Fine level: ws[p] = weight of edge (i,j)-(i+1,j), we[p] = weight of edge
// (i,j)-(i,j+1) (zero on the last row / column), ga = diag(A^T A).
template <class T>
struct FineOp {
  int nv, nh;
  const T* __restrict__ ws;
  const T* __restrict__ we;
  const T* __restrict__ ga;

  // (L^T W L z)_p for the value accessor v(q) of one column
  template <class F>
  __device__ __forceinline__ T lap(int64_t p, int i, int j, F v) const {
    const T zp = v(p);
    T acc = 0;
    if (i + 1 < nv) acc += ws[p] * (zp - v(p + 1));
    if (i > 0) acc += ws[p - 1] * (zp - v(p - 1));
    if (j + 1 < nh) acc += we[p] * (zp - v(p + nv));
    if (j > 0) acc += we[p - nv] * (zp - v(p - nv));
    return acc;
  }
  template <class F>
  __device__ __forceinline__ T apply(int64_t p, int i, int j, T lam2, F v) const {
    return lam2 * lap(p, i, j, v) + ga[p] * v(p);
  }
  // the same with the value accessor v(di, dj) of the neighbour at offset
  // (di, dj) (shared-memory tiles)
  static constexpr int kRadius = 1;
  template <class F>
  __device__ __forceinline__ T apply_off(int64_t p, int i, int j, T lam2, F v) const {
    const T zp = v(0, 0);
    T acc = 0;
    if (i + 1 < nv) acc += ws[p] * (zp - v(1, 0));
    if (i > 0) acc += ws[p - 1] * (zp - v(-1, 0));
    if (j + 1 < nh) acc += we[p] * (zp - v(0, 1));
    if (j > 0) acc += we[p - nv] * (zp - v(0, -1));
    return lam2 * acc + ga[p] * zp;
  }
  __device__ __forceinline__ double diagL(int64_t p, int i, int j) const {
    double s = 0;
    if (i + 1 < nv) s += (double)ws[p];
    if (i > 0) s += (double)ws[p - 1];
    if (j + 1 < nh) s += (double)we[p];
    if (j > 0) s += (double)we[p - nv];
    return s;
  }
  // sum_q |k_pq| and k_pp of lam2 G_L + G_A
  __device__ __forceinline__ double l1(int64_t p, int i, int j, double lam2) const {
    return 2.0 * lam2 * diagL(p, i, j) + (double)ga[p];
  }
  __device__ __forceinline__ double center(int64_t p, int i, int j, double lam2) const {
    return lam2 * diagL(p, i, j) + (double)ga[p];
  }
  // enumerate (neighbour, coefficient) of row p of lam2 G_L + G_A
  template <class F>
  __device__ __forceinline__ void row(int64_t p, int i, int j, double lam2, F emit) const {
    emit(p, center(p, i, j, lam2));
    if (i + 1 < nv) emit(p + 1, -lam2 * (double)ws[p]);
    if (i > 0) emit(p - 1, -lam2 * (double)ws[p - 1]);
    if (j + 1 < nh) emit(p + nv, -lam2 * (double)we[p]);
    if (j > 0) emit(p - nv, -lam2 * (double)we[p - nv]);
  }
};

// Coarse level: per point a row of kCoefStride values, the 25 coefficients
// of lam^2-part G_L at [0, 25) and of G_A at [32, 57); the coefficient of
// neighbour (i+di, j+dj) has offset o = (di+2) + 5 (dj+2).  Coefficients of
// neighbours outside the grid are zero.
constexpr int kCoefStride = 64;

template <class T>
struct CoefVec;
template <>
struct CoefVec<float> {
  using V = float4;
  static constexpr int W = 4;
};
template <>
struct CoefVec<double> {
  using V = double2;
  static constexpr int W = 2;
};

template <class T>
__device__ __forceinline__ void vstore(T* dst, const typename CoefVec<T>::V& v);
template <>
__device__ __forceinline__ void vstore<float>(float* d, const float4& v) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }
template <>
__device__ __forceinline__ void vstore<double>(double* d, const double2& v) { d[0] = v.x; d[1] = v.y; }

template <class T>
struct CoarseOp {
  int nv, nh;
  int64_t n;
  const T* __restrict__ cf;  // [n][kCoefStride]

  // k[o] = lam2 G_L[o] + G_A[o] for point p (vector loads)
  __device__ __forceinline__ void coefs(int64_t p, T lam2, T (&k)[28]) const {
    using VT = typename CoefVec<T>::V;
    constexpr int W = CoefVec<T>::W;
    const VT* row = reinterpret_cast<const VT*>(cf + p * kCoefStride);
    T gl[28], ga[28];
#pragma unroll
    for (int q = 0; q < 28 / W; ++q) {
      vstore<T>(gl + q * W, row[q]);
      vstore<T>(ga + q * W, row[32 / W + q]);
    }
#pragma unroll
    for (int o = 0; o < 28; ++o) k[o] = lam2 * gl[o] + ga[o];
  }

  template <class F>
  __device__ __forceinline__ T apply(int64_t p, int i, int j, T lam2, F v) const {
    T k[28];
    coefs(p, lam2, k);
    T acc = 0;
    if (i >= 2 && i + 2 < nv && j >= 2 && j + 2 < nh) {
#pragma unroll
      for (int dj = -2; dj <= 2; ++dj)
#pragma unroll
        for (int di = -2; di <= 2; ++di) acc += k[(di + 2) + 5 * (dj + 2)] * v(p + di + (int64_t)dj * nv);
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
        acc += k[(di + 2) + 5 * (dj + 2)] * v((int64_t)ii + (int64_t)jj * nv);
      }
    }
    return acc;
  }
  static constexpr int kRadius = 2;
  template <class F>
  __device__ __forceinline__ T apply_off(int64_t p, int i, int j, T lam2, F v) const {
    T k[28];
    coefs(p, lam2, k);
    return apply_k(k, i, j, v);
  }
  // the same with the coefficients k of the point already loaded (coefs)
  template <class F>
  __device__ __forceinline__ T apply_k(const T (&k)[28], int i, int j, F v) const {
    T acc = 0;
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
  __device__ __forceinline__ double l1(int64_t p, int i, int j, double lam2) const {
    const T* row = cf + p * kCoefStride;
    double s = 0;
    for (int o = 0; o < kStencil; ++o) s += fabs(lam2 * (double)row[o] + (double)row[32 + o]);
    return s;
  }
  __device__ __forceinline__ double center(int64_t p, int, int, double lam2) const {
    const T* row = cf + p * kCoefStride;
    return lam2 * (double)row[12] + (double)row[32 + 12];
  }
  template <class F>
  __device__ __forceinline__ void row(int64_t p, int i, int j, double lam2, F emit) const {
    const T* rw = cf + p * kCoefStride;
    for (int dj = -2; dj <= 2; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= nh) continue;
      for (int di = -2; di <= 2; ++di) {
        const int ii = i + di;
        if (ii < 0 || ii >= nv) continue;
        const int o = (di + 2) + 5 * (dj + 2);
        emit((int64_t)ii + (int64_t)jj * nv, lam2 * (double)rw[o] + (double)rw[32 + o]);
      }
    }
  }
};

// SoA (25 x n per part, from the Galerkin products) -> AoS rows of the
// smoother; entries 25..31 and 57..63 are zero.
template <class T>
__global__ void k_coef_pack(int64_t n, const double* __restrict__ gl, const double* __restrict__ ga,
                            T* __restrict__ cf) {
  for (int64_t t = (int64_t)blockIdx.x * kBlock + threadIdx.x; t < n * kCoefStride;
       t += (int64_t)gridDim.x * kBlock) {
    const int64_t p = t / kCoefStride;
    const int o = (int)(t - p * kCoefStride);
    double v = 0.0;
    if (o < kStencil) v = gl[(int64_t)o * n + p];
    else if (o >= 32 && o < 32 + kStencil) v = ga[(int64_t)(o - 32) * n + p];
    cf[t] = (T)v;
  }
}

// ---------------------------------------------------------------------------
// Per-column PCG state (device) and the scalar updates that follow the dot
// products.  They run either as their own small kernels or in the last
// block of the kernel that produced the partial sums ("last block done":
// every block writes its partials, fences, takes a ticket; the block that
// takes the final ticket sums all partials in block order, so the result
// does not depend on which block finished last).
// ---------------------------------------------------------------------------
struct ColState {
  double* rz;      // r^T z of the current iterate
  double* rz2;     // the same value, written by every writer of rz; the
                   // one-column fused beta writes rz2 only and the fused
                   // alpha that follows reads rz2 and copies it to rz, so
                   // neither kernel reads a slot it writes
  double* alpha;
  double* beta;
  double* rr;      // ||r||^2 (recursive)
  double* rmax;    // largest ||r||^2 since the last reliable update
  double* tol2cc;  // tol^2 ||c||^2
  int* active;
  int* iters;
  int* status;
  int* pending;    // recursive residual reached tol: true residual needed
  int* counters;   // [0] active columns, [1] pending columns, [2] reliable-update votes
  int keep;        // 1: a column whose true residual fails the check continues
                   // from its current search direction (residual replacement);
                   // 0: it restarts with p = z
};

// The recursive residual of column col reached tol: the column waits for
// its true-residual check.  With st.keep its beta and rz advance as in a
// regular step (k_update_p then forms p = z + beta p for it), so that a
// failed check continues CG from that direction with the residual replaced.
__device__ __forceinline__ void mark_pending(const ColState& st, int col, double rzn) {
  st.pending[col] = 1;
  st.active[col] = 0;
  if (st.keep && rzn > 0.0) {
    st.beta[col] = rzn / st.rz[col];
    st.rz[col] = rzn;
    st.rz2[col] = rzn;
  } else {
    st.beta[col] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// CSR SpMM over B interleaved columns.  One warp per row; the 32 lanes are
// S = 32/G nnz-groups x G column groups of CPG columns each, so a lane
// reads one (value, column) pair and CPG consecutive vector entries per
// step; the S partial sums are combined with xor shuffles.
//   MODE 0: Y[r] = (A X)[r]
//   MODE 1: Q[r] = (A^T Y)[r] + lam2 (L^T W L P)[r], dot partials of P.Q
//           (rows are pixels; X = Y of the first stage)
//   MODE 2: partials of ||(A X)[r] - b[r]||^2   (residual norm rho)
//   MODE 3: R[r] = C[r] - ((A^T Y)[r] + lam2 (L^T W L P)[r] + 0), partials
//           of R.R   (true residual of the normal equations)
// ---------------------------------------------------------------------------
struct SpmmArgs {
  int64_t rows;
  const int64_t* rp;
  const int32_t* ci;
  int B;        // leading dimension (columns) of every batched vector
  int c0;       // first column handled by this launch (blockIdx.y adds chunks)
  int nb;       // columns in [c0, c0 + nb) are handled
  int nl;       // MODE 2: lambdas per right-hand side (b column = col / nl)
  int nrhs;     // MODE 2: columns of b
  int variant;            // one-column kernel (k_spmv1): 0 = the pass's default,
                          // 1 = 32 lanes x 4, 2 = 16 lanes x 8, 3 = 8 lanes x 8;
                          // FP32 vectors only (else as 3): 4 = 8 x 8 with at
                          // least 5 blocks per SM, 5 = 8 x 8 with 6, 6 = 8 x 4
                          // with 8
  // one-column kernel: column of nonzero k of row r = rbase[r] + c16[k]
  // (null: ci), 6 instead of 8 bytes per FP32 nonzero
  const uint16_t* c16;
  const int32_t* rbase;
};

template <class V, class T, class TO, int G, int CPG, int MODE>
__global__ void __launch_bounds__(kBlock)
    k_spmm(SpmmArgs a, const V* __restrict__ va, const T* __restrict__ X, TO* __restrict__ Y,
           FineOp<T> fop, const T* __restrict__ P, const T* __restrict__ C,
           const double* __restrict__ lam2, const double* __restrict__ bvec,
           double* __restrict__ part) {
  constexpr int S = 32 / G;
  __shared__ double sdot[kBlock / 32][G * CPG];
  const int lane = threadIdx.x & 31, warp_in_block = threadIdx.x >> 5;
  const int g = lane % G, s = lane / G;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
  const int cfirst = a.c0 + blockIdx.y * (G * CPG);
  const int cend = min(a.c0 + a.nb, cfirst + G * CPG);
  const int cbase = cfirst + g * CPG;
  double dacc[CPG];
#pragma unroll
  for (int t = 0; t < CPG; ++t) dacc[t] = 0.0;

  constexpr int U = 4;  // nonzeros per lane in flight
  for (int64_t r = warp; r < a.rows; r += nwarps) {
    const int64_t k0 = a.rp[r], k1 = a.rp[r + 1];
    T acc[CPG];
#pragma unroll
    for (int t = 0; t < CPG; ++t) acc[t] = 0;
    for (int64_t kb = k0 + s; kb < k1; kb += S * U) {
      // the matrix is streamed once per apply: load it evict-first so the
      // gathered vectors stay in L2; all loads of the step are independent
      int cu[U];
      T vu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = kb + (int64_t)u * S;
        const bool ok = k < k1;
        cu[u] = ok ? __ldcs(a.ci + k) : 0;
        vu[u] = ok ? (T)__ldcs(va + k) : (T)0;
      }
      T xv[U][CPG];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const T* xr = X + (int64_t)cu[u] * a.B + cbase;
#pragma unroll
        for (int t = 0; t < CPG; ++t) xv[u][t] = (cbase + t < cend) ? xr[t] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int t = 0; t < CPG; ++t) acc[t] += vu[u] * xv[u][t];
    }
#pragma unroll
    for (int off = G; off < 32; off <<= 1)
#pragma unroll
      for (int t = 0; t < CPG; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], off);
    if (s == 0) {
      int i = 0, j = 0;
      if (MODE == 1 || MODE == 3) {
        j = (int)(r / fop.nv);
        i = (int)(r - (int64_t)j * fop.nv);
      }
#pragma unroll
      for (int t = 0; t < CPG; ++t) {
        const int col = cbase + t;
        if (col >= cend) continue;
        if (MODE == 0) {
          Y[r * a.B + col] = (TO)acc[t];
        } else if (MODE == 1 || MODE == 3) {
          auto pv = [&](int64_t q) { return P[q * a.B + col]; };
          const T lap = fop.lap(r, i, j, pv);
          const T qv = acc[t] + (T)lam2[col] * lap;
          if (MODE == 1) {
            Y[r * a.B + col] = (TO)qv;
            dacc[t] += to_d(P[r * a.B + col]) * to_d(qv);
          } else {
            const T rv = C[r * a.B + col] - qv;
            Y[r * a.B + col] = (TO)rv;
            dacc[t] += to_d(rv) * to_d(rv);
          }
        } else {  // MODE 2
          const double e = to_d(acc[t]) - bvec[r * a.nrhs + col / a.nl];
          dacc[t] += e * e;
        }
      }
    }
  }
  if (MODE != 0) {
    // lanes s == 0 hold the column-group sums of their warp
    if (s == 0) {
#pragma unroll
      for (int t = 0; t < CPG; ++t) sdot[warp_in_block][g * CPG + t] = dacc[t];
    }
    __syncthreads();
    const int width = cend - cfirst;
    if ((int)threadIdx.x < width) {
      double sum = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) sum += sdot[w][threadIdx.x];
      part[(int64_t)blockIdx.x * a.B + cfirst + threadIdx.x] = sum;
    }
  }
}

// ---------------------------------------------------------------------------
// One column (a batch of B = 1, the paper's warm-start chain).  A row is
// handled by LPR lanes, so a warp works on 32 / LPR rows at once; each lane
// keeps U nonzeros in flight, and the row pointers of the warp's next rows
// are loaded before the current rows' gathers (PF).  Same modes as k_spmm.
// Measured on GB300 (256^2 CT, 15M nonzeros): y = A p is fastest with 32
// lanes per row and U = 4; the transposed pass, whose epilogue (L^T W L p
// and p.q) runs on one lane per row, with 8 lanes per row and U = 8.
// C16: column indices as 16-bit offsets from a per-row base (a.c16,
// a.rbase), when every row's column span is below 65,536.
// ---------------------------------------------------------------------------
// MINB: resident blocks per SM the register allocation must allow (the
// launch bound; more blocks = fewer registers per thread).
template <class T, int LPR>
constexpr int spmv1_minb() { return sizeof(T) == 4 ? (LPR == 32 ? 8 : 4) : (LPR == 32 ? 5 : 3); }

template <class V, class T, class TO, int MODE, int U, int LPR, bool PF, bool C16, int MINB>
__global__ void __launch_bounds__(kBlock, MINB)
    k_spmv1(SpmmArgs a, const V* __restrict__ va, const T* __restrict__ X, TO* __restrict__ Y,
            FineOp<T> fop, const T* __restrict__ P, const T* __restrict__ C,
            const double* __restrict__ lam2, const double* __restrict__ bvec,
            double* __restrict__ part) {
  constexpr int RPW = 32 / LPR;  // rows per warp step
  __shared__ double sdot[kBlock / 32];
  const int lane = threadIdx.x & 31;
  const int sl = lane % LPR, hw = lane / LPR;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
  const int64_t ld = a.B;
  const int col = a.c0;
  const T l2 = (MODE == 1 || MODE == 3) ? (T)lam2[col] : (T)0;
  double dacc = 0.0;
  int64_t wr = warp;
  int64_t r = wr * RPW + hw;
  int64_t k0 = 0, k1 = 0;
  int rb = 0;
  if (r < a.rows) {
    k0 = a.rp[r];
    k1 = a.rp[r + 1];
    if (C16) rb = a.rbase[r];
  }
  // every lane of a warp runs the same number of steps (the shuffles below
  // take the whole warp); lanes past the last row compute nothing
  while (wr * RPW < a.rows) {
    const int64_t wrn = wr + nwarps;
    const int64_t rn = wrn * RPW + hw;
    int64_t k0n = 0, k1n = 0;
    int rbn = 0;
    if (PF && rn < a.rows) {
      k0n = a.rp[rn];
      k1n = a.rp[rn + 1];
      if (C16) rbn = a.rbase[rn];
    }
    T acc = 0;
    for (int64_t kb = k0 + sl; kb < k1; kb += LPR * U) {
      // the matrix is streamed once per apply: evict-first loads
      int cu[U];
      T vu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = kb + (int64_t)u * LPR;
        const bool ok = k < k1;
        if (C16)
          cu[u] = ok ? rb + (int)__ldcs(a.c16 + k) : 0;
        else
          cu[u] = ok ? __ldcs(a.ci + k) : 0;
        vu[u] = ok ? (T)__ldcs(va + k) : (T)0;
      }
      T xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = X[(int64_t)cu[u] * ld + col];
#pragma unroll
      for (int u = 0; u < U; ++u) acc += vu[u] * xv[u];
    }
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (sl == 0 && r < a.rows) {
      if (MODE == 0) {
        Y[r * ld + col] = (TO)acc;
      } else if (MODE == 1 || MODE == 3) {
        const int j = (int)(r / fop.nv), i = (int)(r - (int64_t)j * fop.nv);
        auto pv = [&](int64_t q) { return P[q * ld + col]; };
        const T qv = acc + l2 * fop.lap(r, i, j, pv);
        if (MODE == 1) {
          Y[r * ld + col] = (TO)qv;
          dacc += to_d(P[r * ld + col]) * to_d(qv);
        } else {
          const T rv = C[r * ld + col] - qv;
          Y[r * ld + col] = (TO)rv;
          dacc += to_d(rv) * to_d(rv);
        }
      } else {  // MODE 2
        const double e = to_d(acc) - bvec[r * a.nrhs + col / a.nl];
        dacc += e * e;
      }
    }
    wr = wrn;
    r = rn;
    if (PF) {
      k0 = k0n;
      k1 = k1n;
      rb = rbn;
    } else if (r < a.rows) {
      k0 = a.rp[r];
      k1 = a.rp[r + 1];
      if (C16) rb = a.rbase[r];
    }
  }
  if (MODE != 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, off);
    if (lane == 0) sdot[threadIdx.x >> 5] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < kBlock / 32; ++w) sum += sdot[w];
      part[(int64_t)blockIdx.x * ld + col] = sum;
    }
  }
}

constexpr int kCsrPad = 4;  // padding elements after the last nonzero of a CSR array

// ---------------------------------------------------------------------------
// V-cycle level kernels (point x column mapping)
// ---------------------------------------------------------------------------
// dinv = 1 / sum_q |k_pq| (l1-Jacobi) or omega / k_pp (damped Jacobi)
template <class Op, class T>
__global__ void __launch_bounds__(kBlock)
    k_dinv(Op op, int64_t n, int B, const double* __restrict__ lam2, int smoother, double omega,
           T* __restrict__ dinv) {
  const ColMap cm(B);
  if (!cm.ok) return;
  for (int64_t p = cm.first(); p < n; p += cm.stride()) {
    const int j = (int)(p / op.nv), i = (int)(p - (int64_t)j * op.nv);
    const double l2 = lam2[cm.col];
    const double v = smoother == 0 ? 1.0 / op.l1(p, i, j, l2) : omega / op.center(p, i, j, l2);
    dinv[p * B + cm.col] = (T)v;
  }
}

// Pre-smoothing from a zero initial guess: one sweep gives z = dinv r; two
// sweeps give z = z1 + dinv (r - K z1) with z1 = dinv r formed on the fly.
template <class Op, class T>
__global__ void __launch_bounds__(kBlock)
    k_smooth_zero(Op op, int64_t n, int B, const T* __restrict__ lam2, const T* __restrict__ dinv,
                  const T* __restrict__ r, T* __restrict__ z, int two) {
  const ColMap cm(B);
  if (!cm.ok) return;
  const int col = cm.col;
  const T l2 = lam2[col];
  for (int64_t p = cm.first(); p < n; p += cm.stride()) {
    const T z1 = dinv[p * B + col] * r[p * B + col];
    if (!two) {
      z[p * B + col] = z1;
      continue;
    }
    const int j = (int)(p / op.nv), i = (int)(p - (int64_t)j * op.nv);
    auto v = [&](int64_t q) { return dinv[q * B + col] * r[q * B + col]; };
    const T kz = op.apply(p, i, j, l2, v);
    z[p * B + col] = z1 + dinv[p * B + col] * (r[p * B + col] - kz);
  }
}

// One Jacobi-type sweep zout = zin + dinv (r - K zin); optionally the
// partials of r . zout per column.
template <class Op, class T>
__global__ void __launch_bounds__(kBlock)
    k_smooth(Op op, int64_t n, int B, const T* __restrict__ lam2, const T* __restrict__ dinv,
             const T* __restrict__ r, const T* __restrict__ zin, T* __restrict__ zout,
             const int* __restrict__ active, double* __restrict__ part) {
  __shared__ double sm[kBlock];
  const ColMap cm(B);
  DotAcc<T> dacc;
  if (cm.ok) {
    const int col = cm.col;
    const T l2 = lam2[col];
    for (int64_t p = cm.first(); p < n; p += cm.stride()) {
      const int j = (int)(p / op.nv), i = (int)(p - (int64_t)j * op.nv);
      auto v = [&](int64_t q) { return zin[q * B + col]; };
      const T kz = op.apply(p, i, j, l2, v);
      const T rv = r[p * B + col];
      const T zn = zin[p * B + col] + dinv[p * B + col] * (rv - kz);
      zout[p * B + col] = zn;
      dacc.add(rv, zn);
    }
  }
  if (part) block_col_sum(dacc.value(), cm, sm, part + (int64_t)blockIdx.x * B);
}

// res = r - K z
template <class Op, class T>
__global__ void __launch_bounds__(kBlock)
    k_residual(Op op, int64_t n, int B, const T* __restrict__ lam2, const T* __restrict__ r,
               const T* __restrict__ z, T* __restrict__ res) {
  const ColMap cm(B);
  if (!cm.ok) return;
  const int col = cm.col;
  const T l2 = lam2[col];
  for (int64_t p = cm.first(); p < n; p += cm.stride()) {
    const int j = (int)(p / op.nv), i = (int)(p - (int64_t)j * op.nv);
    auto v = [&](int64_t q) { return z[q * B + col]; };
    res[p * B + col] = r[p * B + col] - op.apply(p, i, j, l2, v);
  }
}

// rc = P^T res_f  (R = P^T, Sec. 3.1)
template <class T>
__global__ void __launch_bounds__(kBlock)
    k_restrict(int nvc, int nhc, int B, const T* __restrict__ rf, T* __restrict__ rc) {
  const ColMap cm(B);
  if (!cm.ok) return;
  const int col = cm.col;
  const int nvf = 2 * nvc, nhf = 2 * nhc;
  const int64_t nc = (int64_t)nvc * nhc;
  for (int64_t p = cm.first(); p < nc; p += cm.stride()) {
    const int J = (int)(p / nvc), I = (int)(p - (int64_t)J * nvc);
    T acc = 0;
#pragma unroll
    for (int b = 2 * J - 1; b <= 2 * J + 2; ++b) {
      if (b < 0 || b >= nhf) continue;
      const T wb = pw1<T>(b, J, nhc);
#pragma unroll
      for (int a2 = 2 * I - 1; a2 <= 2 * I + 2; ++a2) {
        if (a2 < 0 || a2 >= nvf) continue;
        acc += wb * pw1<T>(a2, I, nvc) * rf[((int64_t)a2 + (int64_t)b * nvf) * B + col];
      }
    }
    rc[p * B + col] = acc;
  }
}

// z_f += P e_c
template <class T>
__global__ void __launch_bounds__(kBlock)
    k_prolong_add(int nvc, int nhc, int B, const T* __restrict__ ec, T* __restrict__ zf) {
  const ColMap cm(B);
  if (!cm.ok) return;
  const int col = cm.col;
  const int nvf = 2 * nvc;
  const int64_t nf = (int64_t)nvf * 2 * nhc;
  for (int64_t p = cm.first(); p < nf; p += cm.stride()) {
    const int b = (int)(p / nvf), a2 = (int)(p - (int64_t)b * nvf);
    const int I0 = a2 >> 1, J0 = b >> 1;
    const int I1 = (a2 & 1) ? I0 + 1 : I0 - 1;
    const int J1 = (b & 1) ? J0 + 1 : J0 - 1;
    T acc = 0;
    const int Is[2] = {I0, I1}, Js[2] = {J0, J1};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int J = Js[u];
      if (J < 0 || J >= nhc) continue;
      const T wb = pw1<T>(b, J, nhc);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int I = Is[t];
        if (I < 0 || I >= nvc) continue;
        acc += wb * pw1<T>(a2, I, nvc) * ec[((int64_t)I + (int64_t)J * nvc) * B + col];
      }
    }
    zf[p * B + col] += acc;
  }
}

// ---------------------------------------------------------------------------
// Coarsest level: e = K_c(lam)^{-1} r with the explicit inverse (FP64).
// Block (x, col) computes rows 8x .. 8x + 7 of column col, one warp per row.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kBlock)
    k_coarse_solve(int nc, int B, const double* __restrict__ kinv, const T* __restrict__ rc,
                   T* __restrict__ ec) {
  extern __shared__ double rs[];
  const int col = blockIdx.y;
  for (int q = threadIdx.x; q < nc; q += kBlock) rs[q] = to_d(rc[(int64_t)q * B + col]);
  __syncthreads();
  const double* M = kinv + (int64_t)col * nc * nc;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    const int i = blockIdx.x * (kBlock / 32) + w;
    if (i >= nc) return;
    double s = 0.0;
    for (int q = lane; q < nc; q += 32) s += M[(int64_t)i * nc + q] * rs[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) ec[(int64_t)i * B + col] = from_d<T>(s);
  }
}

// Assemble the dense K_c(lam) = lam^2 G_L + G_A of the coarsest level for
// every column: M[col][p][q].  M must be zeroed first.
template <class Op>
__global__ void __launch_bounds__(kBlock)
    k_dense_assemble(Op op, int64_t n, int B, const double* __restrict__ lam2,
                     double* __restrict__ M) {
  const ColMap cm(B);
  if (!cm.ok) return;
  for (int64_t p = cm.first(); p < n; p += cm.stride()) {
    const int j = (int)(p / op.nv), i = (int)(p - (int64_t)j * op.nv);
    double* row = M + ((int64_t)cm.col * n + p) * n;
    op.row(p, i, j, lam2[cm.col], [&](int64_t q, double k) { row[q] += k; });
  }
}

// In-place dense Cholesky K = L L^T (lower, row-major) followed by the
// explicit inverse K^{-1} = L^{-T} L^{-1}; one block per column.  W is an
// n x n scratch per column.  info[col] = 0 on success, else the 1-based
// pivot that was not positive.
static __global__ void __launch_bounds__(kBlock)
    k_cholesky_inverse(int n, double* __restrict__ Mall, double* __restrict__ Wall,
                       double* __restrict__ Kall, int* __restrict__ info) {
  const int col = blockIdx.x;
  double* M = Mall + (int64_t)col * n * n;
  double* X = Wall + (int64_t)col * n * n;
  double* K = Kall + (int64_t)col * n * n;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = M[(int64_t)k * n + k];
      if (!(d > 0.0) && !bad) bad = k + 1;
      M[(int64_t)k * n + k] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double piv = M[(int64_t)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += kBlock) M[(int64_t)i * n + k] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += kBlock) {
      const int i = k + 1 + (int)(t / m), jj = k + 1 + (int)(t % m);
      if (jj <= i) M[(int64_t)i * n + jj] -= M[(int64_t)i * n + k] * M[(int64_t)jj * n + k];
    }
    __syncthreads();
  }
  // X = L^{-1} (lower): column c by forward substitution, one thread per c
  for (int c = threadIdx.x; c < n; c += kBlock) {
    for (int i = 0; i < c; ++i) X[(int64_t)i * n + c] = 0.0;
    for (int i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= M[(int64_t)i * n + k] * X[(int64_t)k * n + c];
      X[(int64_t)i * n + c] = s / M[(int64_t)i * n + i];
    }
  }
  __syncthreads();
  // K^{-1}[p][q] = sum_{i >= max(p,q)} X[i][p] X[i][q]
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += kBlock) {
    const int p = (int)(t / n), q = (int)(t % n);
    if (q < p) continue;
    double s = 0.0;
    for (int i = q; i < n; ++i) s += X[(int64_t)i * n + p] * X[(int64_t)i * n + q];
    K[(int64_t)p * n + q] = s;
    K[(int64_t)q * n + p] = s;
  }
  if (threadIdx.x == 0) info[col] = bad;
}

// ---------------------------------------------------------------------------
// Galerkin coarse operators G_c = P^T G_f P (Sec. 3.1), one thread per
// (coarse point, stencil offset).  The fine operator is either the level-0
// 5-point L^T W L (part 0), the level-0 diagonal diag(A^T A) (part 1), or a
// 25-point coarse stencil (part 2).
// ---------------------------------------------------------------------------
struct RapIn {
  int part;
  int nvf, nhf;
  int64_t nf;
  const double* ws;
  const double* we;
  const double* ga;
  const double* g25;
  __device__ __forceinline__ double coef(int di, int dj, int64_t f, int fi, int fj) const {
    if (part == 2) return g25[((di + 2) + 5 * (dj + 2)) * nf + f];
    if (part == 1) return (di == 0 && dj == 0) ? ga[f] : 0.0;
    // part 0: L^T W L
    if (di == 0 && dj == 0) {
      double s = 0;
      if (fi + 1 < nvf) s += ws[f];
      if (fi > 0) s += ws[f - 1];
      if (fj + 1 < nhf) s += we[f];
      if (fj > 0) s += we[f - nvf];
      return s;
    }
    if (dj == 0 && di == 1) return -ws[f];
    if (dj == 0 && di == -1) return -ws[f - 1];
    if (di == 0 && dj == 1) return -we[f];
    if (di == 0 && dj == -1) return -we[f - nvf];
    return 0.0;
  }
};

static __global__ void __launch_bounds__(kBlock) k_galerkin(RapIn in, int nvc, int nhc, double* __restrict__ out) {
  const int64_t nc = (int64_t)nvc * nhc;
  const int R = (in.part == 2) ? 2 : 1;
  for (int64_t t = (int64_t)blockIdx.x * kBlock + threadIdx.x; t < nc * kStencil;
       t += (int64_t)gridDim.x * kBlock) {
    const int o = (int)(t / nc);
    const int64_t P = t - (int64_t)o * nc;
    const int J = (int)(P / nvc), I = (int)(P - (int64_t)J * nvc);
    const int oi = o % 5 - 2, oj = o / 5 - 2;
    const int It = I + oi, Jt = J + oj;
    double sum = 0.0;
    if (It >= 0 && It < nvc && Jt >= 0 && Jt < nhc) {
      for (int b = 2 * J - 1; b <= 2 * J + 2; ++b) {
        if (b < 0 || b >= in.nhf) continue;
        const double wb = pw1(b, J, nhc);
        for (int a = 2 * I - 1; a <= 2 * I + 2; ++a) {
          if (a < 0 || a >= in.nvf) continue;
          const double wab = wb * pw1(a, I, nvc);
          const int64_t f = (int64_t)a + (int64_t)b * in.nvf;
          for (int dj = -R; dj <= R; ++dj) {
            const int d = b + dj;
            if (d < 0 || d >= in.nhf) continue;
            const double wd = pw1(d, Jt, nhc);
            if (wd == 0.0) continue;
            for (int di = -R; di <= R; ++di) {
              const int c = a + di;
              if (c < 0 || c >= in.nvf) continue;
              if (in.part != 2 && di != 0 && dj != 0) continue;
              const double wc = pw1(c, It, nvc);
              if (wc == 0.0) continue;
              sum += wab * in.coef(di, dj, f, a, b) * wc * wd;
            }
          }
        }
      }
    }
    out[t] = sum;
  }
}

// ---------------------------------------------------------------------------
// PCG recurrences.  Per-column scalars live in device memory; a column
// whose active flag is 0 is frozen (converged, stopped, or waiting for its
// true-residual check) and left unchanged.
// ---------------------------------------------------------------------------
// x += alpha p ; r -= alpha q ; partials of r.r
template <class T, class TX>
__global__ void __launch_bounds__(kBlock)
    k_update_xr(int64_t n, int B, ColState st, const T* __restrict__ p, const T* __restrict__ q,
                TX* __restrict__ x, T* __restrict__ r, double* __restrict__ part) {
  __shared__ double sm[kBlock];
  const ColMap cm(B);
  DotAcc<T> acc;
  if (cm.ok && st.active[cm.col]) {
    const int col = cm.col;
    const double al = st.alpha[col];
    const T alT = (T)al;
    for (int64_t i = cm.first(); i < n; i += cm.stride()) {
      const int64_t e = i * B + col;
      x[e] = (TX)(x[e] + (TX)al * (TX)p[e]);
      const T rn = r[e] - alT * q[e];
      r[e] = rn;
      acc.add(rn, rn);
    }
  }
  block_col_sum(acc.value(), cm, sm, part + (int64_t)blockIdx.x * B);
}

// The sum of nb partials in a fixed order (the same in every block), by the
// block's first warp; valid in lane 0 of warp 0 only.  One warp keeps the
// FP64 work per block to nb additions: on this GPU the FP64 pipe runs at a
// small fraction of the FP32 one, and every block of the fused updates
// repeats the sum.
__device__ __forceinline__ double warp0_sum(const double* __restrict__ part, int nb) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += part[b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// One column (B = 1) with alpha taken in the update: every block sums the
// p.q partials in the same fixed order, so all blocks compute the same
// alpha = rz / p.q (rz read from the rz2 slot) and the same breakdown
// decision; block 0 alone records the column state (iteration count,
// status, rz = rz2) and clears the counters the beta step accumulates.  No
// block reads what block 0 writes, and block 0 writes active = 0 only when
// every block has found the step void.
template <class T, class TX>
__global__ void __launch_bounds__(kBlock)
    k_update_xr_alpha(int64_t n, ColState st, int nb_pq, const double* __restrict__ pq_part,
                      const T* __restrict__ p, const T* __restrict__ q, TX* __restrict__ x, T* __restrict__ r,
                      double* __restrict__ part) {
  __shared__ double s_al;
  __shared__ int s_ok;
  __shared__ double sm[kBlock / 32];
  double pq = 0.0;
  if (threadIdx.x < 32) pq = warp0_sum(pq_part, nb_pq);
  const int act = st.active[0];
  const double rzc = st.rz2[0];
  const bool fin = isfinite(pq);
  if (threadIdx.x == 0) {  // the step length once per block
    s_ok = act && fin && pq > 0.0;
    s_al = s_ok ? rzc / pq : 0.0;
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  const double al = s_al;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st.rz[0] = rzc;
    st.counters[0] = 0;
    st.counters[1] = 0;
    st.counters[2] = 0;
    st.alpha[0] = al;
    if (act) {
      st.iters[0] += 1;
      if (!fin) {
        st.status[0] = ST_NONFINITE;
        st.active[0] = 0;
      } else if (!(pq > 0.0)) {
        st.status[0] = ST_BREAKDOWN;
        st.active[0] = 0;
      }
    }
  }
  DotAcc<T> dacc;
  if (ok) {
    const T alT = (T)al;
    const TX alX = (TX)al;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
      x[i] = (TX)(x[i] + alX * (TX)p[i]);
      const T rn = r[i] - alT * q[i];
      r[i] = rn;
      dacc.add(rn, rn);
    }
  }
  double acc = dacc.value();
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
}


// One column (B = 1, st.keep = 0) with beta taken in the p update: every
// block sums the r.r and r.z partials in the same fixed order and takes the
// same decision as k_scalar_col_beta (non-finite, converged -> true-residual
// check, iteration limit, breakdown, or a regular step with
// beta = rz_new / rz); only a regular step updates p = z + beta p.  Block 0
// alone writes the column state; the new rz goes to the rz2 slot (the fused
// alpha of the next iteration reads it there and copies it to rz), so no
// block reads a value written in this kernel, and block 0 clears active
// only when every block has found no regular step.
template <class T>
__global__ void __launch_bounds__(kBlock)
    k_update_p_beta(int64_t n, ColState st, int nb_rr, const double* __restrict__ rr_part, int nb_rz,
                    const double* __restrict__ rz_part, int maxit, double rel_trigger, const T* __restrict__ z,
                    T* __restrict__ p) {
  __shared__ double s_be;
  __shared__ int s_kind;
  double rr = 0.0, rzn = 0.0;
  if (threadIdx.x < 32) {
    rr = warp0_sum(rr_part, nb_rr);
    rzn = warp0_sum(rz_part, nb_rz);
  }
  const int act = st.active[0];
  if (threadIdx.x == 0) {  // the decision and beta once per block
    int kd = -1;  // -1 inactive, 0 regular, 1 converged, 2 limit, 3 breakdown, 4 non-finite
    if (act) {
      if (!isfinite(rr) || !isfinite(rzn)) kd = 4;
      else if (rr <= st.tol2cc[0]) kd = 1;
      else if (st.iters[0] >= maxit) kd = 2;
      else if (!(rzn > 0.0)) kd = 3;
      else kd = 0;
    }
    s_kind = kd;
    s_be = kd == 0 ? rzn / st.rz[0] : 0.0;
  }
  __syncthreads();
  const int kind = s_kind;
  const double be = s_be;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (act) {
      st.rr[0] = rr;
      if (kind == 0) {
        st.beta[0] = be;
        st.rz2[0] = rzn;
        if (rel_trigger > 0.0 && rr < rel_trigger * st.rmax[0]) atomicAdd(&st.counters[2], 1);
      } else {
        st.beta[0] = 0.0;
        st.active[0] = 0;
        if (kind == 1) st.pending[0] = 1;
        if (kind == 2) st.status[0] = ST_MAXIT;
        if (kind == 3) st.status[0] = ST_BREAKDOWN;
        if (kind == 4) st.status[0] = ST_NONFINITE;
      }
    }
    if (st.active[0]) atomicAdd(&st.counters[0], 1);
    if (st.pending[0]) atomicAdd(&st.counters[1], 1);
  }
  if (kind == 0) {
    const T bT = (T)be;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
      p[i] = z[i] + bT * p[i];
  }
}

// p = z + beta p
template <class T>
__global__ void __launch_bounds__(kBlock)
    k_update_p(int64_t n, int B, ColState st, const T* __restrict__ z, T* __restrict__ p) {
  const ColMap cm(B);
  if (!cm.ok || !(st.active[cm.col] || (st.keep && st.pending[cm.col]))) return;
  const int col = cm.col;
  const T be = (T)st.beta[col];
  for (int64_t i = cm.first(); i < n; i += cm.stride()) {
    const int64_t e = i * B + col;
    p[e] = z[e] + be * p[e];
  }
}

// restart for the flagged columns: p = z (and the caller sets rz)
template <class T>
__global__ void __launch_bounds__(kBlock)
    k_copy_cols(int64_t n, int B, const int* __restrict__ flag, const T* __restrict__ src,
                T* __restrict__ dst) {
  const ColMap cm(B);
  if (!cm.ok || (flag && !flag[cm.col])) return;
  for (int64_t i = cm.first(); i < n; i += cm.stride()) dst[i * B + cm.col] = src[i * B + cm.col];
}

// Scalar kernels run as one block of kScalarThreads threads: warp w sums
// the block partials of columns w, w + 32, ... with a fixed lane stride and
// shuffle tree (deterministic), and lane 0 applies the per-column update.
constexpr int kScalarThreads = 1024;

__device__ __forceinline__ double warp_sum_parts(const double* part, int nblk, int B, int col) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * B + col];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// serial form for callers that are one thread per column
__device__ __forceinline__ double sum_parts(const double* part, int nblk, int B, int col) {
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * B + col];
  return s;
}

// One block of kColThreads threads per column sums that column's partials
// (fixed thread stride and tree: deterministic) so the FP64 additions are
// spread over B multiprocessors.
constexpr int kColThreads = 512;

__device__ __forceinline__ double block_sum_parts(const double* part, int nblk, int B, int col) {
  __shared__ double sm[kColThreads / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kColThreads) s += part[(int64_t)b * B + col];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kColThreads / 32; ++w) t += sm[w];
  return t;
}

// alpha = rz / p^T q ; grid = B blocks.  Also clears the counters that
// k_scalar_col_beta accumulates.
static __global__ void __launch_bounds__(kColThreads)
    k_scalar_col_alpha(int B, int nblk, const double* __restrict__ pq_part, ColState st) {
  const int col = blockIdx.x;
  if (col == 0 && threadIdx.x < 3) st.counters[threadIdx.x] = 0;
  if (!st.active[col]) {
    if (threadIdx.x == 0) st.alpha[col] = 0.0;
    return;
  }
  const double pq = block_sum_parts(pq_part, nblk, B, col);
  if (threadIdx.x != 0) return;
  st.iters[col] += 1;
  if (!isfinite(pq)) {
    st.status[col] = ST_NONFINITE;
    st.active[col] = 0;
    st.alpha[col] = 0.0;
  } else if (!(pq > 0.0)) {
    st.status[col] = ST_BREAKDOWN;
    st.active[col] = 0;
    st.alpha[col] = 0.0;
  } else {
    st.alpha[col] = st.rz[col] / pq;
  }
}

// rr, recursive convergence and beta for one column per block; counters
// (cleared by k_scalar_col_alpha) accumulate with integer atomics.
static __global__ void __launch_bounds__(kColThreads)
    k_scalar_col_beta(int B, int nblk_rr, const double* __restrict__ rr_part, int nblk_rz,
                      const double* __restrict__ rz_part, ColState st, int maxit, double rel_trigger) {
  const int col = blockIdx.x;
  if (st.active[col]) {
    const double rr = block_sum_parts(rr_part, nblk_rr, B, col);
    const double rzn = block_sum_parts(rz_part, nblk_rz, B, col);
    if (threadIdx.x == 0) {
      st.rr[col] = rr;
      if (!isfinite(rr) || !isfinite(rzn)) {
        st.status[col] = ST_NONFINITE;
        st.active[col] = 0;
        st.beta[col] = 0.0;
      } else if (rr <= st.tol2cc[col]) {
        mark_pending(st, col, rzn);
      } else if (st.iters[col] >= maxit) {
        st.status[col] = ST_MAXIT;
        st.active[col] = 0;
        st.beta[col] = 0.0;
      } else if (!(rzn > 0.0)) {
        st.status[col] = ST_BREAKDOWN;
        st.active[col] = 0;
        st.beta[col] = 0.0;
      } else {
        st.beta[col] = rzn / st.rz[col];
        st.rz[col] = rzn;
        st.rz2[col] = rzn;
        if (rel_trigger > 0.0 && rr < rel_trigger * st.rmax[col]) atomicAdd(&st.counters[2], 1);
      }
    }
  }
  if (threadIdx.x == 0) {
    if (st.active[col]) atomicAdd(&st.counters[0], 1);
    if (st.pending[col]) atomicAdd(&st.counters[1], 1);
  }
}



// Sum partials of a column reduction into out[col] (FP64).
static __global__ void __launch_bounds__(kScalarThreads)
    k_sum_parts(int B, int nblk, const double* __restrict__ part, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int col = w; col < B; col += kScalarThreads / 32) {
    const double s = warp_sum_parts(part, nblk, B, col);
    if (lane == 0) out[col] = s;
  }
}

// ---------------------------------------------------------------------------
// Element-wise helpers
// ---------------------------------------------------------------------------
// dst[p][j] = src[p][j / per] (expand per-right-hand-side data to columns)
template <class TS, class TD>
__global__ void k_expand_cols(int64_t n, int B, int per, int nsrc, const TS* __restrict__ src,
                              TD* __restrict__ dst) {
  const ColMap cm(B);
  if (!cm.ok) return;
  for (int64_t i = cm.first(); i < n; i += cm.stride())
    dst[i * B + cm.col] = (TD)src[i * nsrc + cm.col / per];
}

// convert / copy with type change
template <class TS, class TD>
__global__ void k_convert(int64_t count, const TS* __restrict__ src, TD* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < count; i += (int64_t)gridDim.x * kBlock)
    dst[i] = (TD)src[i];
}

// planar [B][n] <-> interleaved [n][B]
static __global__ void k_planar_to_inter(int64_t n, int B, const double* __restrict__ src, double* __restrict__ dst) {
  const ColMap cm(B);
  if (!cm.ok) return;
  for (int64_t i = cm.first(); i < n; i += cm.stride()) dst[i * B + cm.col] = src[(int64_t)cm.col * n + i];
}
static __global__ void k_inter_to_planar(int64_t n, int B, const double* __restrict__ src, double* __restrict__ dst) {
  const ColMap cm(B);
  if (!cm.ok) return;
  for (int64_t i = cm.first(); i < n; i += cm.stride()) dst[(int64_t)cm.col * n + i] = src[i * B + cm.col];
}

// dst[i][j] = src_j[i] for planar column pointers src_j (null -> 0)
static __global__ void k_gather_cols(int64_t n, int B, const double* const* __restrict__ src,
                                     double* __restrict__ dst) {
  const ColMap cm(B);
  if (!cm.ok) return;
  const double* s = src[cm.col];
  for (int64_t i = cm.first(); i < n; i += cm.stride()) dst[i * B + cm.col] = s ? s[i] : 0.0;
}

// dst_j[i] = src[i][j] for non-null planar column pointers dst_j
static __global__ void k_scatter_cols(int64_t n, int B, const double* __restrict__ src,
                                      double* const* __restrict__ dst) {
  const ColMap cm(B);
  if (!cm.ok) return;
  double* d = dst[cm.col];
  if (!d) return;
  for (int64_t i = cm.first(); i < n; i += cm.stride()) d[i] = src[i * B + cm.col];
}

// dst[i][j] = src[i][map[j]] (src has nsrc columns)
static __global__ void k_gather_map(int64_t n, int B, int nsrc, const int* __restrict__ map,
                                    const double* __restrict__ src, double* __restrict__ dst) {
  const ColMap cm(B);
  if (!cm.ok) return;
  const int sc = map[cm.col];
  for (int64_t i = cm.first(); i < n; i += cm.stride()) dst[i * B + cm.col] = src[i * nsrc + sc];
}

static __global__ void k_negate(int64_t count, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < count; i += (int64_t)gridDim.x * kBlock)
    x[i] = -x[i];
}

// x64 += (double) xlo ; xlo = 0   (reliable update of the mixed path)
static __global__ void k_flush_x(int64_t count, float* __restrict__ xlo, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < count; i += (int64_t)gridDim.x * kBlock) {
    x[i] += (double)xlo[i];
    xlo[i] = 0.0f;
  }
}

// column sums of squares over the rows of A^T: diag(A^T A)
template <class V>
__global__ void k_diag_ata(int64_t n, const int64_t* __restrict__ rpT, const V* __restrict__ vT,
                           double* __restrict__ diag) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kBlock) >> 5;
  for (int64_t r = warp; r < n; r += nw) {
    double s = 0.0;
    for (int64_t k = rpT[r] + lane; k < rpT[r + 1]; k += 32) {
      const double v = (double)vT[k];
      s += v * v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) diag[r] = s;
  }
}

// edge weights d -> per-pixel squared weights ws, we
static __global__ void k_edge_to_pixel(int nv, int nh, const double* __restrict__ d, double* __restrict__ ws,
                                double* __restrict__ we) {
  const int64_t n = (int64_t)nv * nh;
  const int64_t nvert = (int64_t)nh * (nv - 1);
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    const int j = (int)(p / nv), i = (int)(p - (int64_t)j * nv);
    double a = 0.0, b = 0.0;
    if (i + 1 < nv) {
      const double v = d[i + (int64_t)j * (nv - 1)];
      a = v * v;
    }
    if (j + 1 < nh) {
      const double v = d[nvert + i + (int64_t)j * nv];
      b = v * v;
    }
    ws[p] = a;
    we[p] = b;
  }
}

// eta^2 partials: ||D L x||^2 = sum ws (x_{p+1}-x_p)^2 + we (x_{p+nv}-x_p)^2
static __global__ void __launch_bounds__(kBlock)
    k_seminorm(int nv, int nh, int B, const double* __restrict__ ws, const double* __restrict__ we,
               const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sm[kBlock];
  const ColMap cm(B);
  const int64_t n = (int64_t)nv * nh;
  double acc = 0.0;
  if (cm.ok) {
    for (int64_t p = cm.first(); p < n; p += cm.stride()) {
      const int j = (int)(p / nv), i = (int)(p - (int64_t)j * nv);
      const double xp = x[p * B + cm.col];
      if (i + 1 < nv) {
        const double t = x[(p + 1) * B + cm.col] - xp;
        acc += ws[p] * t * t;
      }
      if (j + 1 < nh) {
        const double t = x[(p + nv) * B + cm.col] - xp;
        acc += we[p] * t * t;
      }
    }
  }
  block_col_sum(acc, cm, sm, part + (int64_t)blockIdx.x * B);
}

// weight update (eq. (g)): stage 1 writes |v_e| = |d_e (L x)_e| and block maxima
static __global__ void k_weighted_grad(int nv, int nh, const double* __restrict__ d, const double* __restrict__ x,
                                double* __restrict__ absv, double* __restrict__ bmax) {
  __shared__ double sm[kBlock];
  const int64_t nvert = (int64_t)nh * (nv - 1);
  const int64_t ne = nvert + (int64_t)(nh - 1) * nv;
  double m = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < ne; e += (int64_t)gridDim.x * kBlock) {
    double g;
    if (e < nvert) {
      const int64_t j = e / (nv - 1), i = e - j * (nv - 1);
      const int64_t p = i + j * nv;
      g = x[p + 1] - x[p];
    } else {
      const int64_t f = e - nvert;
      const int64_t j = f / nv, i = f - j * nv;
      const int64_t p = i + j * nv;
      g = x[p + nv] - x[p];
    }
    const double v = fabs(d[e] * g);
    absv[e] = v;
    m = fmax(m, v);
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = kBlock / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) bmax[blockIdx.x] = sm[0];
}

// stage 2: d <- max(1 - (|v|/vmax)^q, d_min) d   (unchanged if vmax == 0)
static __global__ void k_weight_apply(int64_t ne, int nblk, const double* __restrict__ bmax,
                               const double* __restrict__ absv, double q, double d_min,
                               double* __restrict__ d) {
  __shared__ double vmax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int b = 0; b < nblk; ++b) m = fmax(m, bmax[b]);
    vmax = m;
  }
  __syncthreads();
  if (vmax == 0.0) return;
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < ne; e += (int64_t)gridDim.x * kBlock) {
    const double g = absv[e] / vmax;
    const double gq = (q == 2.0) ? g * g : (q == 1.0 ? g : pow(g, q));
    d[e] = fmax(1.0 - gq, d_min) * d[e];
  }
}

// partials of x . y per column
template <class T>
__global__ void __launch_bounds__(kBlock)
    k_col_dot(int64_t n, int B, const T* __restrict__ x, const T* __restrict__ y, double* __restrict__ part) {
  __shared__ double sm[kBlock];
  const ColMap cm(B);
  DotAcc<T> acc;
  if (cm.ok)
    for (int64_t i = cm.first(); i < n; i += cm.stride()) acc.add(x[i * B + cm.col], y[i * B + cm.col]);
  block_col_sum(acc.value(), cm, sm, part + (int64_t)blockIdx.x * B);
}

// start of a solve: per-column state from ||c||^2 and the true residual
static __global__ void k_init_state(int B, double tol, const double* __restrict__ cc, const double* __restrict__ rr,
                             ColState st) {
  const int col = threadIdx.x;
  if (col >= B) return;
  st.tol2cc[col] = tol * tol * cc[col];
  st.iters[col] = 0;
  st.pending[col] = 0;
  st.rr[col] = rr[col];
  st.rmax[col] = rr[col];
  st.alpha[col] = 0.0;
  st.beta[col] = 0.0;
  if (!isfinite(rr[col])) {
    st.status[col] = ST_NONFINITE;
    st.active[col] = 0;
  } else if (rr[col] <= st.tol2cc[col]) {
    st.status[col] = ST_CONVERGED;
    st.active[col] = 0;
  } else {
    st.status[col] = ST_RUNNING;
    st.active[col] = 1;
  }
}

// True-residual check / reliable update.  flag[col]: 1 = restart (pending
// column whose true residual is still above tol), 2 = replace the residual
// of a running column (mixed path), 0 = leave.
static __global__ void k_true_check(int B, const double* __restrict__ rr_true, ColState st, int replace_active,
                             int* __restrict__ flag) {
  __shared__ int cnt[2];
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int col = threadIdx.x;
  if (col < B) {
    int f = 0;
    const double rr = rr_true[col];
    if (st.pending[col]) {
      st.pending[col] = 0;
      if (rr <= st.tol2cc[col]) {
        st.status[col] = ST_CONVERGED;
      } else if (!isfinite(rr)) {
        st.status[col] = ST_NONFINITE;
      } else {
        st.active[col] = 1;
        st.rmax[col] = rr;
        st.rr[col] = rr;
        f = st.keep ? 2 : 1;  // 2: replace the residual only; 1: also restart
      }
    } else if (st.active[col] && replace_active) {
      st.rmax[col] = rr;
      st.rr[col] = rr;
      f = 2;
    }
    flag[col] = f;
    if (st.active[col]) atomicAdd(&cnt[0], 1);
    if (f == 1) atomicAdd(&cnt[1], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st.counters[0] = cnt[0];
    st.counters[1] = 0;
    st.counters[2] = 0;
    st.counters[3] = cnt[1];
  }
}

// r[:, col] = (T) r64[:, col] for flagged columns
template <class T>
__global__ void k_take_residual(int64_t n, int B, const int* __restrict__ flag, const double* __restrict__ r64,
                                T* __restrict__ r) {
  const ColMap cm(B);
  if (!cm.ok || !flag[cm.col]) return;
  for (int64_t i = cm.first(); i < n; i += cm.stride()) r[i * B + cm.col] = (T)r64[i * B + cm.col];
}

// after a restart V-cycle: rz = r.z and p = z for restarted columns
template <class T>
__global__ void k_restart_finish(int64_t n, int B, int nblk, const double* __restrict__ part,
                                 const int* __restrict__ flag, ColState st, const T* __restrict__ z,
                                 T* __restrict__ p) {
  const ColMap cm(B);
  if (!cm.ok || flag[cm.col] != 1) return;
  if (blockIdx.x == 0 && cm.k == 0) st.rz[cm.col] = st.rz2[cm.col] = sum_parts(part, nblk, B, cm.col);
  for (int64_t i = cm.first(); i < n; i += cm.stride()) p[i * B + cm.col] = z[i * B + cm.col];
}

// zero every column of a batch whose flag is set (c = 0 systems)
static __global__ void k_zero_cols(int64_t n, int B, const double* __restrict__ cc, double* __restrict__ x) {
  const ColMap cm(B);
  if (!cm.ok || cc[cm.col] != 0.0) return;
  for (int64_t i = cm.first(); i < n; i += cm.stride()) x[i * B + cm.col] = 0.0;
}

// ---------------------------------------------------------------------------
// Blur forward operator: zero-boundary correlation with a kh x kw PSF.
//   (A x)(i, j) = sum_{u,v} psf[u + rv][v + rh] x(i + u, j + v)
//   (A^T y)(i, j) = sum_{u,v} psf[u + rv][v + rh] y(i - u, j - v)
// ---------------------------------------------------------------------------
struct PsfArgs {
  int nv, nh, rv, rh;   // radii: kh = 2 rv + 1, kw = 2 rh + 1
  const double* psf;    // row-major kh x kw
};

template <class T, int TRANS>
__device__ __forceinline__ T psf_apply(const PsfArgs& a, const T* __restrict__ psf, int64_t p, int i, int j,
                                       const T* __restrict__ x, int B, int col) {
  const int kw = 2 * a.rh + 1;
  T acc = 0;
  for (int v = -a.rh; v <= a.rh; ++v) {
    const int jj = TRANS ? j - v : j + v;
    if (jj < 0 || jj >= a.nh) continue;
    for (int u = -a.rv; u <= a.rv; ++u) {
      const int ii = TRANS ? i - u : i + u;
      if (ii < 0 || ii >= a.nv) continue;
      acc += psf[(u + a.rv) * kw + (v + a.rh)] * x[((int64_t)ii + (int64_t)jj * a.nv) * B + col];
    }
  }
  return acc;
}

// y = A x (MODE 0) or partials of ||A x - b||^2 (MODE 2)
template <class T, int MODE>
__global__ void __launch_bounds__(kBlock)
    k_psf_forward(PsfArgs a, const T* __restrict__ psf, int B, const T* __restrict__ x, T* __restrict__ y,
                  const double* __restrict__ bvec, int nl, int nrhs, double* __restrict__ part) {
  __shared__ double sm[kBlock];
  const ColMap cm(B);
  const int64_t n = (int64_t)a.nv * a.nh;
  double acc = 0.0;
  if (cm.ok) {
    for (int64_t p = cm.first(); p < n; p += cm.stride()) {
      const int j = (int)(p / a.nv), i = (int)(p - (int64_t)j * a.nv);
      const T v = psf_apply<T, 0>(a, psf, p, i, j, x, B, cm.col);
      if (MODE == 0) {
        y[p * B + cm.col] = v;
      } else {
        const double e = to_d(v) - bvec[p * nrhs + cm.col / nl];
        acc += e * e;
      }
    }
  }
  if (MODE == 2) block_col_sum(acc, cm, sm, part + (int64_t)blockIdx.x * B);
}

// q = A^T y + lam2 L^T W L p with partials of p.q (MODE 1), or
// r = c - (A^T y + lam2 L^T W L p) with partials of r.r (MODE 3)
template <class T, class TO, int MODE>
__global__ void __launch_bounds__(kBlock)
    k_psf_normal(PsfArgs a, const T* __restrict__ psf, int B, const T* __restrict__ y, FineOp<T> fop,
                 const T* __restrict__ P, const T* __restrict__ C, const double* __restrict__ lam2,
                 TO* __restrict__ out, double* __restrict__ part) {
  __shared__ double sm[kBlock];
  const ColMap cm(B);
  const int64_t n = (int64_t)a.nv * a.nh;
  DotAcc<T> acc;
  if (cm.ok) {
    const int col = cm.col;
    const T l2 = (T)lam2[col];
    for (int64_t p = cm.first(); p < n; p += cm.stride()) {
      const int j = (int)(p / a.nv), i = (int)(p - (int64_t)j * a.nv);
      const T aty = psf_apply<T, 1>(a, psf, p, i, j, y, B, col);
      auto pv = [&](int64_t q) { return P[q * B + col]; };
      const T qv = aty + l2 * fop.lap(p, i, j, pv);
      if (MODE == 1) {
        out[p * B + col] = (TO)qv;
        acc.add(P[p * B + col], qv);
      } else {
        const T rv = C[p * B + col] - qv;
        out[p * B + col] = (TO)rv;
        acc.add(rv, rv);
      }
    }
  }
  block_col_sum(acc.value(), cm, sm, part + (int64_t)blockIdx.x * B);
}

// c = A^T b for the n_rhs right-hand sides (interleaved [n][nrhs])
static __global__ void k_psf_rhs(PsfArgs a, int nrhs, const double* __restrict__ b, double* __restrict__ c) {
  const ColMap cm(nrhs);
  if (!cm.ok) return;
  const int64_t n = (int64_t)a.nv * a.nh;
  for (int64_t p = cm.first(); p < n; p += cm.stride()) {
    const int j = (int)(p / a.nv), i = (int)(p - (int64_t)j * a.nv);
    c[p * nrhs + cm.col] = psf_apply<double, 1>(a, a.psf, p, i, j, b, nrhs, cm.col);
  }
}

// diag(A^T A)_p = sum of psf^2 over offsets whose row p - (u, v) is inside
static __global__ void k_psf_diag(PsfArgs a, double* __restrict__ diag) {
  const int64_t n = (int64_t)a.nv * a.nh;
  const int kw = 2 * a.rh + 1;
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    const int j = (int)(p / a.nv), i = (int)(p - (int64_t)j * a.nv);
    double s = 0.0;
    for (int v = -a.rh; v <= a.rh; ++v) {
      const int jj = j - v;
      if (jj < 0 || jj >= a.nh) continue;
      for (int u = -a.rv; u <= a.rv; ++u) {
        const int ii = i - u;
        if (ii < 0 || ii >= a.nv) continue;
        const double w = a.psf[(u + a.rv) * kw + (v + a.rh)];
        s += w * w;
      }
    }
    diag[p] = s;
  }
}


}  // namespace lcmg
