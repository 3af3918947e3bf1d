// Device kernels of the paper's own preconditioner (Sec. 3.2-3.3) and its
// flexible GMRES: one column, FP64.
//
// Level k applies K_k x = A_k^T (A_k x) + lam2 M_k^T (M_k x) in three
// launches: y = A_k x and t = A_k^T y with the CSR SpMV kernels, then
// k_pm_lap_add adds lam2 M_k^T M_k x, where M_k^T M_k = G_L^k is the
// Galerkin coarsening of L^T D^2 L (the 5-point fine operator on level 0;
// on coarser levels the 25-point stencils of the geometric hierarchy or the
// CSR matrices of classical AMG).  Relaxation is Jacobi-
// preconditioned CG; its scalar recurrences are taken by every block from
// the previous kernel's block partials (summed in a fixed order, so every
// block computes the same alpha and beta and no scalar kernel or host
// round trip is needed).
#pragma once
#include "kernels.cuh"

namespace lcmg {

// 25-point Galerkin stencil of L^T D^2 L on a coarse level, stored as
// 25 x n arrays (offset o = (di + 2) + 5 (dj + 2)).
struct GLOp {
  int nv, nh;
  int64_t n;
  const double* __restrict__ gl;
  template <class F>
  __device__ __forceinline__ double lap(int64_t p, int i, int j, F v) const {
    double acc = 0.0;
#pragma unroll
    for (int dj = -2; dj <= 2; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= nh) continue;
#pragma unroll
      for (int di = -2; di <= 2; ++di) {
        const int ii = i + di;
        if (ii < 0 || ii >= nv) continue;
        acc += gl[(int64_t)((di + 2) + 5 * (dj + 2)) * n + p] * v((int64_t)ii + (int64_t)jj * nv);
      }
    }
    return acc;
  }
  __device__ __forceinline__ double diagL(int64_t p, int, int) const { return gl[(int64_t)12 * n + p]; }
};

// G_L^k of a classical AMG level: an unstructured CSR matrix (columns
// sorted) with its diagonal.  nv = n, so a point's (i, j) is (p, 0).
struct CsrGLOp {
  int nv;
  int64_t n;
  const int64_t* __restrict__ rp;
  const int32_t* __restrict__ ci;
  const double* __restrict__ v;
  const double* __restrict__ dg;
  template <class F>
  __device__ __forceinline__ double lap(int64_t p, int, int, F x) const {
    double acc = 0.0;
    for (int64_t k = rp[p]; k < rp[p + 1]; ++k) acc += v[k] * x((int64_t)ci[k]);
    return acc;
  }
  __device__ __forceinline__ double diagL(int64_t p, int, int) const { return dg[p]; }
};

// sum of the first nb block partials, in index order (every block gets the
// same value)
__device__ __forceinline__ double pm_sum_parts(const double* __restrict__ part, int nb, double* sm) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += kBlock) s += part[b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kBlock / 32; ++w) t += sm[w];
  __syncthreads();
  return t;
}

// block partial of v over the block's points
__device__ __forceinline__ void pm_block_part(double v, double* sm, double* part) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sm[w];
    part[blockIdx.x] = t;
  }
}

// s = t + lam2 (M^T M x)_p; MODE 0: q = s with partials of x.q;
// MODE 1: q = b - s (a residual), no partials
template <class Op, int MODE>
__global__ void __launch_bounds__(kBlock)
    k_pm_lap_add(Op op, int64_t n, const double* __restrict__ lam2, const double* __restrict__ x,
                 const double* __restrict__ t, const double* __restrict__ b, double* __restrict__ q,
                 double* __restrict__ part) {
  __shared__ double sm[kBlock / 32];
  const double l2 = lam2[0];
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    const int j = (int)(p / op.nv), i = (int)(p - (int64_t)j * op.nv);
    auto v = [&](int64_t k) { return x[k]; };
    const double s = t[p] + l2 * op.lap(p, i, j, v);
    if (MODE == 0) {
      q[p] = s;
      acc += x[p] * s;
    } else {
      q[p] = b[p] - s;
    }
  }
  if (MODE == 0) pm_block_part(acc, sm, part);
}

// dinv = 1 / (diag(A^T A) + lam2 diag(M^T M))
template <class Op>
__global__ void __launch_bounds__(kBlock)
    k_pm_dinv(Op op, int64_t n, const double* __restrict__ lam2, const double* __restrict__ dA,
              double* __restrict__ dinv) {
  const double l2 = lam2[0];
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    const int j = (int)(p / op.nv), i = (int)(p - (int64_t)j * op.nv);
    dinv[p] = 1.0 / (dA[p] + l2 * op.diagL(p, i, j));
  }
}

// start of a relaxation call: r = b (zero_x: x = 0) or r as given;
// z = dinv r, p = z, partials of r.z
__global__ void __launch_bounds__(kBlock)
    k_pm_cg_init(int64_t n, int zero_x, const double* __restrict__ b, const double* __restrict__ dinv,
                 double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                 double* __restrict__ p, double* __restrict__ part_rz) {
  __shared__ double sm[kBlock / 32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    double ri;
    if (zero_x) {
      x[i] = 0.0;
      ri = b[i];
      r[i] = ri;
    } else {
      ri = r[i];
    }
    const double zi = dinv[i] * ri;
    z[i] = zi;
    p[i] = zi;
    acc += ri * zi;
  }
  pm_block_part(acc, sm, part_rz);
}

// alpha = (r.z) / (p.q) from the partials; x += alpha p; r -= alpha q;
// z = dinv r; partials of the new r.z.  alpha = 0 when either sum is not
// positive (the step is skipped, as the CG breakdown rule).
__global__ void __launch_bounds__(kBlock)
    k_pm_cg_xr(int64_t n, const double* __restrict__ part_rz, int nb_rz, const double* __restrict__ part_pq,
               int nb_pq, const double* __restrict__ p, const double* __restrict__ q,
               const double* __restrict__ dinv, double* __restrict__ x, double* __restrict__ r,
               double* __restrict__ z, double* __restrict__ part_rz_new) {
  __shared__ double sm[kBlock / 32];
  const double rz = pm_sum_parts(part_rz, nb_rz, sm);
  const double pq = pm_sum_parts(part_pq, nb_pq, sm);
  const double a = (rz > 0.0 && pq > 0.0) ? rz / pq : 0.0;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    x[i] += a * p[i];
    const double ri = r[i] - a * q[i];
    r[i] = ri;
    const double zi = dinv[i] * ri;
    z[i] = zi;
    acc += ri * zi;
  }
  pm_block_part(acc, sm, part_rz_new);
}

// beta = (r.z)_new / (r.z)_old; p = z + beta p (beta = 0 if the old sum is
// not positive)
__global__ void __launch_bounds__(kBlock)
    k_pm_cg_p(int64_t n, const double* __restrict__ part_new, const double* __restrict__ part_old, int nb,
              const double* __restrict__ z, double* __restrict__ p) {
  __shared__ double sm[kBlock / 32];
  const double rn = pm_sum_parts(part_new, nb, sm);
  const double ro = pm_sum_parts(part_old, nb, sm);
  const double be = ro > 0.0 ? rn / ro : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
    p[i] = z[i] + be * p[i];
}

// dense K_c = A_c^T A_c + lam2 G_L^c of the coarsest level (row-major),
// one thread per entry: the stencil coefficient of row p at column q when
// q lies within the 5 x 5 neighbourhood of p
__global__ void __launch_bounds__(kBlock)
    k_pm_dense(GLOp op, const double* __restrict__ lam2, const double* __restrict__ AtA,
               double* __restrict__ M) {
  const int64_t n = op.n;
  const double l2 = lam2[0];
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * kBlock) {
    const int64_t p = e / n, q = e - p * n;
    const int pj = (int)(p / op.nv), pi = (int)(p - (int64_t)pj * op.nv);
    const int qj = (int)(q / op.nv), qi = (int)(q - (int64_t)qj * op.nv);
    const int di = qi - pi, dj = qj - pj;
    double v = AtA[e];
    if (di >= -2 && di <= 2 && dj >= -2 && dj <= 2)
      v += l2 * op.gl[(int64_t)((di + 2) + 5 * (dj + 2)) * n + p];
    M[e] = v;
  }
}

// dense K_c = A_c^T A_c + lam2 G_L^c from the dense G_L^c of a classical
// AMG coarsest level (nn = n_c^2 entries)
__global__ void __launch_bounds__(kBlock)
    k_pm_dense_add(int64_t nn, const double* __restrict__ lam2, const double* __restrict__ AtA,
                   const double* __restrict__ G, double* __restrict__ M) {
  const double l2 = lam2[0];
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < nn; e += (int64_t)gridDim.x * kBlock)
    M[e] = AtA[e] + l2 * G[e];
}

// y = M x (ADD: y += M x) for a CSR matrix M of `rows` rows: the
// restriction P^T r and the prolongation x += P e of classical AMG levels;
// one thread per row (P has a few entries per row)
template <bool ADD>
__global__ void __launch_bounds__(kBlock)
    k_pm_csr_mv(int64_t rows, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t r = (int64_t)blockIdx.x * kBlock + threadIdx.x; r < rows; r += (int64_t)gridDim.x * kBlock) {
    double acc = 0.0;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) acc += v[k] * x[ci[k]];
    y[r] = ADD ? y[r] + acc : acc;
  }
}

// ---- flexible GMRES (Arnoldi with block Gram-Schmidt) ------------------
// part[i][blk] = sum over the block's points of V[i][p] w[p], i < m
__global__ void __launch_bounds__(kBlock)
    k_pm_multidot(int64_t n, int m, const double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                  double* __restrict__ part) {
  __shared__ double sm[kBlock / 32];
  const int i = blockIdx.y;
  const double* vi = V + (int64_t)i * ldv;
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock)
    acc += vi[p] * w[p];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kBlock / 32; ++k) t += sm[k];
    part[(int64_t)i * gridDim.x + blockIdx.x] = t;
  }
  (void)m;
}

// h[i] (+)= sum of part[i][0 .. nb); one warp per i
__global__ void __launch_bounds__(kBlock)
    k_pm_sum_rows(int m, int nb, const double* __restrict__ part, double* __restrict__ h, int accumulate) {
  const int lane = threadIdx.x & 31;
  for (int i = (int)(blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5)); i < m; i += (int)(gridDim.x * (kBlock / 32))) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[(int64_t)i * nb + b];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) h[i] = accumulate ? h[i] + s : s;
  }
}

// w -= sum_i h[i] V[i]  (i < m)
__global__ void __launch_bounds__(kBlock)
    k_pm_orth(int64_t n, int m, const double* __restrict__ V, int64_t ldv, const double* __restrict__ h,
              double* __restrict__ w) {
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    double s = w[p];
    for (int i = 0; i < m; ++i) s -= h[i] * V[(int64_t)i * ldv + p];
    w[p] = s;
  }
}

// x += sum_i y[i] Z[i]  (i < m)
__global__ void __launch_bounds__(kBlock)
    k_pm_combine(int64_t n, int m, const double* __restrict__ Z, int64_t ldz, const double* __restrict__ y,
                 double* __restrict__ x) {
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    double s = x[p];
    for (int i = 0; i < m; ++i) s += y[i] * Z[(int64_t)i * ldz + p];
    x[p] = s;
  }
}

// y = s x
__global__ void __launch_bounds__(kBlock)
    k_pm_scale(int64_t n, double s, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock)
    y[p] = s * x[p];
}

}  // namespace lcmg
