// The finest level of the V(1,1) cycle (Algorithm 1, nu = 1) in two
// kernels, for the mixed path's FP32 vectors.
//
// With one sweep, pre-smoothing from a zero initial guess is z1 = D^{-1} r,
// so the pre-smoothed vector need not be stored: the down kernel forms it
// on the fly for the residual and the restriction, and the up kernel forms
// it again (the same values, the same formulas) under the prolongated
// correction.  D^{-1} (l1-Jacobi 1 / sum_q |k_pq|, or damped Jacobi
// omega / k_pp) is computed from the level's stored weights where it is
// needed, so the level reads r, its weights and the coarse correction and
// writes the coarse right-hand side and z, and nothing else:
//
//   k_vfine_down: z1 = D^{-1} r, res = r - K z1, r_c = P^T res
//   k_vfine_up:   z0 = z1 + P e_c, z = z0 + D^{-1} (r - K z0), partials r.z
//
// A block owns a 64 x 32 tile of fine points (a 32 x 16 tile of coarse
// points) and keeps the windows its stencils need in shared memory
// (halo 2 for the down kernel, 1 for the up kernel); blocks stride over the
// tiles.  The sums per point are those of the generic tile kernels.
#pragma once
#include "compact.cuh"
#include "kernels.cuh"

namespace lcmg {

constexpr int kFineTI = 64;  // fine points per tile along i (contiguous)
constexpr int kFineTJ = 32;  // ... along j
constexpr int kFineThreads = 256;

// the stored fine-level weights of either operator form
__device__ __forceinline__ float fw_s(const FineOp<float>& op, int64_t p) { return op.ws[p]; }
__device__ __forceinline__ float fw_e(const FineOp<float>& op, int64_t p) { return op.we[p]; }
__device__ __forceinline__ float fw_g(const FineOp<float>& op, int64_t p) { return op.ga[p]; }
__device__ __forceinline__ float fw_s(const FineOpH& op, int64_t p) { return op.ws_(p); }
__device__ __forceinline__ float fw_e(const FineOpH& op, int64_t p) { return op.we_(p); }
__device__ __forceinline__ float fw_g(const FineOpH& op, int64_t p) { return op.ga_(p); }

// the four edge weights around point (i, j) (zero across the boundary) and
// diag(A^T A) there
struct FineW {
  float s, n, e, w, g;
};
template <class Op>
__device__ __forceinline__ FineW fine_w(const Op& op, int64_t p, int i, int j) {
  FineW f;
  f.s = i + 1 < op.nv ? fw_s(op, p) : 0.f;
  f.n = i > 0 ? fw_s(op, p - 1) : 0.f;
  f.e = j + 1 < op.nh ? fw_e(op, p) : 0.f;
  f.w = j > 0 ? fw_e(op, p - op.nv) : 0.f;
  f.g = fw_g(op, p);
  return f;
}

// D^{-1} at a point: l1-Jacobi 1 / (2 lam2 sum w + ga), or omega / (lam2 sum w + ga)
__device__ __forceinline__ float fine_dinv(const FineW& f, float l2, int smoother, float omega) {
  const float sw = f.s + f.n + f.e + f.w;
  return smoother == 0 ? 1.0f / (2.0f * l2 * sw + f.g) : omega / (l2 * sw + f.g);
}

// (K z)_p with z read at offsets of a shared-memory window (stride ld)
__device__ __forceinline__ float fine_kz(const FineW& f, float l2, const float* z, int q, int ld) {
  const float zp = z[q];
  const float acc = f.s * (zp - z[q + 1]) + f.n * (zp - z[q - 1]) + f.e * (zp - z[q + ld]) + f.w * (zp - z[q - ld]);
  return l2 * acc + f.g * zp;
}

template <class Op>
__global__ void __launch_bounds__(kFineThreads)
    k_vfine_down(Op op, int B, const float* __restrict__ lam2, int smoother, float omega,
                 const float* __restrict__ r, float* __restrict__ rc, int ntiles) {
  constexpr int ZI = kFineTI + 4, ZJ = kFineTJ + 4;  // z1 window, halo 2
  constexpr int RI = kFineTI + 2, RJ = kFineTJ + 2;  // residual window, halo 1
  __shared__ float sz[ZI * ZJ];
  __shared__ float sr[ZI * ZJ];
  __shared__ float sres[RI * RJ];
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  const int nti = (nv + kFineTI - 1) / kFineTI;
  const float l2 = lam2[col];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = (tile % nti) * kFineTI, j0 = (tile / nti) * kFineTJ;
    // z1 = D^{-1} r and r on the window (zero outside the grid)
    for (int t = threadIdx.x; t < ZI * ZJ; t += kFineThreads) {
      const int i = i0 - 2 + t % ZI, j = j0 - 2 + t / ZI;
      float zv = 0.f, rv = 0.f;
      if (i >= 0 && i < nv && j >= 0 && j < nh) {
        const int64_t p = (int64_t)i + (int64_t)j * nv;
        rv = r[p * B + col];
        zv = fine_dinv(fine_w(op, p, i, j), l2, smoother, omega) * rv;
      }
      sz[t] = zv;
      sr[t] = rv;
    }
    __syncthreads();
    // res = r - K z1
    for (int t = threadIdx.x; t < RI * RJ; t += kFineThreads) {
      const int li = t % RI, lj = t / RI;
      const int i = i0 - 1 + li, j = j0 - 1 + lj;
      float v = 0.f;
      if (i >= 0 && i < nv && j >= 0 && j < nh) {
        const int64_t p = (int64_t)i + (int64_t)j * nv;
        const int q = (li + 1) + (lj + 1) * ZI;
        v = sr[q] - fine_kz(fine_w(op, p, i, j), l2, sz, q, ZI);
      }
      sres[t] = v;
    }
    __syncthreads();
    // r_c = P^T res over the tile's coarse points
    for (int t = threadIdx.x; t < (kFineTI / 2) * (kFineTJ / 2); t += kFineThreads) {
      const int I = i0 / 2 + t % (kFineTI / 2), J = j0 / 2 + t / (kFineTI / 2);
      if (I >= nvc || J >= nhc) continue;
      float acc = 0.f;
#pragma unroll
      for (int b = 2 * J - 1; b <= 2 * J + 2; ++b) {
        if (b < 0 || b >= nh) continue;
        const float wb = pw1<float>(b, J, nhc);
#pragma unroll
        for (int a2 = 2 * I - 1; a2 <= 2 * I + 2; ++a2) {
          if (a2 < 0 || a2 >= nv) continue;
          acc += wb * pw1<float>(a2, I, nvc) * sres[(a2 - (i0 - 1)) + (b - (j0 - 1)) * RI];
        }
      }
      rc[((int64_t)I + (int64_t)J * nvc) * B + col] = acc;
    }
    __syncthreads();  // the windows are refilled by the next tile
  }
}

template <class Op>
__global__ void __launch_bounds__(kFineThreads)
    k_vfine_up(Op op, int B, const float* __restrict__ lam2, int smoother, float omega,
               const float* __restrict__ r, const float* __restrict__ ec, float* __restrict__ zout, int ntiles,
               double* __restrict__ part) {
  constexpr int WI = kFineTI + 2, WJ = kFineTJ + 2;          // z0 window, halo 1
  constexpr int CI = kFineTI / 2 + 2, CJ = kFineTJ / 2 + 2;  // coarse window
  __shared__ float sc[CI * CJ];
  __shared__ float s0[WI * WJ];
  __shared__ double sred[kFineThreads / 32];
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  const int nti = (nv + kFineTI - 1) / kFineTI;
  const float l2 = lam2[col];
  Dot2 dot;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = (tile % nti) * kFineTI, j0 = (tile / nti) * kFineTJ;
    const int I0 = i0 / 2 - 1, J0 = j0 / 2 - 1;
    for (int t = threadIdx.x; t < CI * CJ; t += kFineThreads) {
      const int I = I0 + t % CI, J = J0 + t / CI;
      sc[t] = (I >= 0 && I < nvc && J >= 0 && J < nhc) ? ec[((int64_t)I + (int64_t)J * nvc) * B + col] : 0.f;
    }
    __syncthreads();
    // z0 = D^{-1} r + P e_c on the window
    for (int t = threadIdx.x; t < WI * WJ; t += kFineThreads) {
      const int a2 = i0 - 1 + t % WI, b = j0 - 1 + t / WI;
      float v = 0.f;
      if (a2 >= 0 && a2 < nv && b >= 0 && b < nh) {
        const int64_t p = (int64_t)a2 + (int64_t)b * nv;
        const float z1 = fine_dinv(fine_w(op, p, a2, b), l2, smoother, omega) * r[p * B + col];
        const int Ia = a2 >> 1, Ja = b >> 1;
        const int Ib = (a2 & 1) ? Ia + 1 : Ia - 1;
        const int Jb = (b & 1) ? Ja + 1 : Ja - 1;
        const int Is[2] = {Ia, Ib}, Js[2] = {Ja, Jb};
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int J = Js[u];
          if (J < 0 || J >= nhc) continue;
          const float wb = pw1<float>(b, J, nhc);
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            const int I = Is[w];
            if (I < 0 || I >= nvc) continue;
            acc += wb * pw1<float>(a2, I, nvc) * sc[(I - I0) + (J - J0) * CI];
          }
        }
        v = z1 + acc;
      }
      s0[t] = v;
    }
    __syncthreads();
    // z = z0 + D^{-1} (r - K z0) on the tile's points
    for (int t = threadIdx.x; t < kFineTI * kFineTJ; t += kFineThreads) {
      const int li = t % kFineTI, lj = t / kFineTI;
      const int i = i0 + li, j = j0 + lj;
      if (i >= nv || j >= nh) continue;
      const int64_t p = (int64_t)i + (int64_t)j * nv;
      const FineW f = fine_w(op, p, i, j);
      const int q = (li + 1) + (lj + 1) * WI;
      const float rv = r[p * B + col];
      const float zn = s0[q] + fine_dinv(f, l2, smoother, omega) * (rv - fine_kz(f, l2, s0, q, WI));
      zout[p * B + col] = zn;
      dot.add(rv, zn);
    }
    __syncthreads();
  }
  if (part) {
    double dacc = dot.value();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, off);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < kFineThreads / 32; ++k) s += sred[k];
      part[(int64_t)blockIdx.x * B + col] = s;
    }
  }
}

}  // namespace lcmg
