// The V-cycle of Algorithm 1 with two kernels per level.
//
// With one kernel per step a level costs six launches (pre-smoothing,
// residual, restriction, prolongation, two post-sweeps), and at one column
// per batch every one of them is a few microseconds of latency for a few
// hundred kilobytes of work.  Here a block owns an 8 x 8 tile of coarse
// points and the 16 x 16 fine points whose parents they are, and keeps the
// tile with the halos its stencils need in shared memory:
//
//   k_vdown: z1 = D r, z = z1 + D (r - K z1) (nu = 2) or z = z1 (nu = 1),
//            res = r - K z, r_c = R res        -> z (pre-smoothed), r_c
//   k_vup:   z0 = z + P e_c, then nu sweeps z <- z + D (r - K z)
//            (and the partials of r.z on the finest level)
//
// Halo points are recomputed by every block that needs them, so blocks
// share nothing but global inputs.  k_vup reads the pre-smoothed z of its
// halo from a buffer it does not write (zpre -> zout), so blocks never
// race.  The arithmetic of every point is that of the one-kernel-per-step
// path (same formulas, same order of the stencil sums).
#pragma once
#include "kernels.cuh"

namespace lcmg {

constexpr int kVTile = 8;  // coarse points per tile side
constexpr int kMaxTileBlocks = 2048;  // grid cap of the tile kernels (rows of their partial sums)
// threads of a tile block: enough for one point per thread in every phase
// (the widest window is 22 x 22 on the 5-point finest level and 26 x 26 on
// the 25-point levels with nu = 2; with nu = 1 the 25-point windows are at
// most 22 x 22); FP64 25-point blocks stay at 512 (their stencil rows need
// more than the 64 registers a 1024-thread block allows), and so do nu = 1
// 25-point blocks, whose second phase's loads are issued before the first
// phase's barrier (registers for the prefetched coefficients)
template <class Op, class T, int NU = 2>
__host__ __device__ constexpr int vtile_threads() {
  return (Op::kRadius == 1 || sizeof(T) == 8 || NU == 1) ? 512 : 1024;
}

// block sum of v into part[blockIdx.x * B + col] (NT threads)
template <int NT>
__device__ __forceinline__ void vblock_sum(double v, double* sred, double* part, int B, int col) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += sred[w];
    part[(int64_t)blockIdx.x * B + col] = s;
  }
}

// k_vdown on tile (tx, ty) of column blockIdx.y
template <class Op, class T, int NU>
__device__ __forceinline__ void vdown_tile(const Op& op, int B, const T* __restrict__ lam2,
                                           const T* __restrict__ dinv, const T* __restrict__ r,
                                           T* __restrict__ zpre, T* __restrict__ rc, int tx, int ty) {
  constexpr int NTD = vtile_threads<Op, T, NU>();
  constexpr int H = Op::kRadius;
  constexpr int WR = 2 * kVTile + 2;                  // restriction window
  constexpr int WZ = WR + 2 * H;                      // z window
  constexpr int W1 = (NU == 2) ? WZ + 2 * H : WZ;     // z1 window
  __shared__ T s1[W1 * W1];
  __shared__ T sz[(NU == 2) ? WZ * WZ : 1];
  __shared__ T sres[WR * WR];
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  const int I0 = tx * kVTile, J0 = ty * kVTile;
  const int ri = 2 * I0 - 1, rj = 2 * J0 - 1;  // window origins (fine coordinates)
  const int zi = ri - H, zj = rj - H;
  const int oi = ri - (W1 - WR) / 2, oj = rj - (W1 - WR) / 2;
  const T l2 = lam2[col];
  auto inside = [&](int i, int j) { return i >= 0 && i < nv && j >= 0 && j < nh; };
  auto gidx = [&](int i, int j) { return ((int64_t)i + (int64_t)j * nv) * B + col; };

  // nu = 1 on the 25-point levels: the residual phase's loads (the point's
  // coefficients and r) do not depend on z1, so they are issued before the
  // first barrier, one residual point per thread
  constexpr bool kPre = (NU == 1 && H == 2);
  static_assert(!kPre || WR * WR <= NTD, "one residual point per thread");
  T kpre[kPre ? 28 : 1];
  T rpre = 0;
  int pi = 0, pj = 0;
  bool phave = false;
  if constexpr (kPre) {
    if ((int)threadIdx.x < WR * WR) {
      pi = ri + (int)threadIdx.x % WR;
      pj = rj + (int)threadIdx.x / WR;
      phave = inside(pi, pj);
      if (phave) {
        const int64_t p = (int64_t)pi + (int64_t)pj * nv;
        op.coefs(p, l2, kpre);
        rpre = r[p * B + col];
      }
    }
  }
  // z1 = D r
  for (int t = threadIdx.x; t < W1 * W1; t += NTD) {
    const int i = oi + t % W1, j = oj + t / W1;
    s1[t] = inside(i, j) ? dinv[gidx(i, j)] * r[gidx(i, j)] : (T)0;
  }
  __syncthreads();
  // z = z1 + D (r - K z1)
  if (NU == 2) {
    for (int t = threadIdx.x; t < WZ * WZ; t += NTD) {
      const int i = zi + t % WZ, j = zj + t / WZ;
      T v = 0;
      if (inside(i, j)) {
        const int64_t p = (int64_t)i + (int64_t)j * nv;
        const int q = (i - oi) + (j - oj) * W1;
        auto v1 = [&](int di, int dj) { return s1[q + di + dj * W1]; };
        const T kz = op.apply_off(p, i, j, l2, v1);
        v = s1[q] + dinv[p * B + col] * (r[p * B + col] - kz);
      }
      sz[t] = v;
    }
    __syncthreads();
  }
  const T* zs = (NU == 2) ? sz : s1;
  constexpr int WS = (NU == 2) ? WZ : W1;
  const int si = (NU == 2) ? zi : oi, sj = (NU == 2) ? zj : oj;
  // res = r - K z on the restriction window
  if constexpr (kPre) {
    if ((int)threadIdx.x < WR * WR) {
      T v = 0;
      if (phave) {
        const int q = (pi - si) + (pj - sj) * WS;
        auto vz = [&](int di, int dj) { return zs[q + di + dj * WS]; };
        v = rpre - op.apply_k(kpre, pi, pj, vz);
      }
      sres[threadIdx.x] = v;
    }
  } else {
    for (int t = threadIdx.x; t < WR * WR; t += NTD) {
      const int i = ri + t % WR, j = rj + t / WR;
      T v = 0;
      if (inside(i, j)) {
        const int64_t p = (int64_t)i + (int64_t)j * nv;
        const int q = (i - si) + (j - sj) * WS;
        auto vz = [&](int di, int dj) { return zs[q + di + dj * WS]; };
        v = r[p * B + col] - op.apply_off(p, i, j, l2, vz);
      }
      sres[t] = v;
    }
  }
  // the pre-smoothed z of the tile's own fine points
  for (int t = threadIdx.x; t < 4 * kVTile * kVTile; t += NTD) {
    const int i = 2 * I0 + t % (2 * kVTile), j = 2 * J0 + t / (2 * kVTile);
    if (i < nv && j < nh) zpre[gidx(i, j)] = zs[(i - si) + (j - sj) * WS];
  }
  __syncthreads();
  // r_c = R res
  for (int t = threadIdx.x; t < kVTile * kVTile; t += NTD) {
    const int I = I0 + t % kVTile, J = J0 + t / kVTile;
    if (I >= nvc || J >= nhc) continue;
    T acc = 0;
#pragma unroll
    for (int b = 2 * J - 1; b <= 2 * J + 2; ++b) {
      if (b < 0 || b >= nh) continue;
      const T wb = pw1<T>(b, J, nhc);
#pragma unroll
      for (int a2 = 2 * I - 1; a2 <= 2 * I + 2; ++a2) {
        if (a2 < 0 || a2 >= nv) continue;
        acc += wb * pw1<T>(a2, I, nvc) * sres[(a2 - ri) + (b - rj) * WR];
      }
    }
    rc[((int64_t)I + (int64_t)J * nvc) * B + col] = acc;
  }
}

// k_vup on tile (tx, ty) of column blockIdx.y; returns the tile's part of r.z
template <class Op, class T, int NU>
__device__ __forceinline__ double vup_tile(const Op& op, int B, const T* __restrict__ lam2,
                                           const T* __restrict__ dinv, const T* __restrict__ r,
                                           const T* __restrict__ ec, const T* __restrict__ zpre,
                                           T* __restrict__ zout, int tx, int ty) {
  constexpr int NTD = vtile_threads<Op, T, NU>();
  constexpr int H = Op::kRadius;
  constexpr int WF = 2 * kVTile;           // the tile's fine points
  constexpr int W0 = WF + 2 * NU * H;      // z0 window
  constexpr int W1 = WF + 2 * H;           // window after the first of two sweeps
  __shared__ T s0[W0 * W0];
  __shared__ T s1[(NU == 2) ? W1 * W1 : 1];
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  const int fi = 2 * tx * kVTile, fj = 2 * ty * kVTile;
  const int oi = fi - NU * H, oj = fj - NU * H;
  const int ai = fi - H, aj = fj - H;
  const T l2 = lam2[col];
  auto inside = [&](int i, int j) { return i >= 0 && i < nv && j >= 0 && j < nh; };

  // nu = 1 on the 25-point levels: the sweep's loads (coefficients, r and
  // the inverse diagonal of the tile's fine points) do not depend on z0, so
  // they are issued before the barrier, one fine point per thread
  constexpr bool kPre = (NU == 1 && H == 2);
  static_assert(!kPre || WF * WF <= NTD, "one fine point per thread");
  T kpre[kPre ? 28 : 1];
  T rpre = 0, dpre = 0;
  int pi = 0, pj = 0;
  bool phave = false;
  if constexpr (kPre) {
    if ((int)threadIdx.x < WF * WF) {
      pi = fi + (int)threadIdx.x % WF;
      pj = fj + (int)threadIdx.x / WF;
      phave = inside(pi, pj);
      if (phave) {
        const int64_t p = (int64_t)pi + (int64_t)pj * nv;
        op.coefs(p, l2, kpre);
        rpre = r[p * B + col];
        dpre = dinv[p * B + col];
      }
    }
  }
  // z0 = z + P e_c
  for (int t = threadIdx.x; t < W0 * W0; t += NTD) {
    const int a2 = oi + t % W0, b = oj + t / W0;
    T v = 0;
    if (inside(a2, b)) {
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
        for (int w = 0; w < 2; ++w) {
          const int I = Is[w];
          if (I < 0 || I >= nvc) continue;
          acc += wb * pw1<T>(a2, I, nvc) * ec[((int64_t)I + (int64_t)J * nvc) * B + col];
        }
      }
      v = zpre[((int64_t)a2 + (int64_t)b * nv) * B + col] + acc;
    }
    s0[t] = v;
  }
  __syncthreads();
  // first of two sweeps
  if (NU == 2) {
    for (int t = threadIdx.x; t < W1 * W1; t += NTD) {
      const int i = ai + t % W1, j = aj + t / W1;
      T v = 0;
      if (inside(i, j)) {
        const int64_t p = (int64_t)i + (int64_t)j * nv;
        const int q = (i - oi) + (j - oj) * W0;
        auto v0 = [&](int di, int dj) { return s0[q + di + dj * W0]; };
        const T kz = op.apply_off(p, i, j, l2, v0);
        v = s0[q] + dinv[p * B + col] * (r[p * B + col] - kz);
      }
      s1[t] = v;
    }
    __syncthreads();
  }
  const T* zs = (NU == 2) ? s1 : s0;
  constexpr int WS = (NU == 2) ? W1 : W0;
  const int si = (NU == 2) ? ai : oi, sj = (NU == 2) ? aj : oj;
  // last sweep on the tile's fine points
  DotAcc<T> dacc;
  if constexpr (kPre) {
    if (phave) {
      const int64_t p = (int64_t)pi + (int64_t)pj * nv;
      const int q = (pi - si) + (pj - sj) * WS;
      auto vz = [&](int di, int dj) { return zs[q + di + dj * WS]; };
      const T kz = op.apply_k(kpre, pi, pj, vz);
      const T zn = zs[q] + dpre * (rpre - kz);
      zout[p * B + col] = zn;
      dacc.add(rpre, zn);
    }
  }
  for (int t = kPre ? WF * WF : (int)threadIdx.x; t < WF * WF; t += NTD) {
    const int i = fi + t % WF, j = fj + t / WF;
    if (!inside(i, j)) continue;
    const int64_t p = (int64_t)i + (int64_t)j * nv;
    const int q = (i - si) + (j - sj) * WS;
    auto vz = [&](int di, int dj) { return zs[q + di + dj * WS]; };
    const T kz = op.apply_off(p, i, j, l2, vz);
    const T rv = r[p * B + col];
    const T zn = zs[q] + dinv[p * B + col] * (rv - kz);
    zout[p * B + col] = zn;
    dacc.add(rv, zn);
  }
  return dacc.value();
}

// Grid-stride over the tiles (any number of them: the grid is capped at
// the blocks resident at once); r.z partials per block.
template <class Op, class T, int NU>
__global__ void __launch_bounds__(vtile_threads<Op, T, NU>())
    k_vdown(Op op, int B, const T* __restrict__ lam2, const T* __restrict__ dinv, const T* __restrict__ r,
            T* __restrict__ zpre, T* __restrict__ rc, int ntx, int ntiles) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    vdown_tile<Op, T, NU>(op, B, lam2, dinv, r, zpre, rc, t % ntx, t / ntx);
    __syncthreads();  // the tile's shared arrays are refilled by the next tile
  }
}

template <class Op, class T, int NU>
__global__ void __launch_bounds__(vtile_threads<Op, T, NU>())
    k_vup(Op op, int B, const T* __restrict__ lam2, const T* __restrict__ dinv, const T* __restrict__ r,
          const T* __restrict__ ec, const T* __restrict__ zpre, T* __restrict__ zout, int ntx, int ntiles,
          double* __restrict__ part) {
  constexpr int NT = vtile_threads<Op, T, NU>();
  __shared__ double sred[NT / 32];
  double dacc = 0.0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    dacc += vup_tile<Op, T, NU>(op, B, lam2, dinv, r, ec, zpre, zout, t % ntx, t / ntx);
    __syncthreads();
  }
  if (part) vblock_sum<NT>(dacc, sred, part, B, blockIdx.y);
}

}  // namespace lcmg
