// Coarse levels of the V(1,1) cycle (Algorithm 1, nu = 1) with FP16 level
// operators (CoarseOpH: 24 FP16 off-diagonal coefficients and an FP32 row
// sum per point), the mixed path's default for batches whose columns share
// one lambda.
//
// The two kernels compute what k_vdown / k_vup compute for this operator
// (same formulas, same order of every sum) on the same 8 x 8 coarse tiles:
//
//   k_vdown_h: z1 = D r, res = r - K z1, r_c = R res      -> z1 (pre-smoothed), r_c
//   k_vup_h:   z0 = z1 + P e_c, z = z0 + D (r - K z0)     -> z, partials of r.z
//
// but stage every input of a tile in shared memory with asynchronous copies
// (cp.async) and keep two tiles in flight: a block issues the copies of its
// next tile before it computes the current one, so the loads of one tile
// overlap the arithmetic of the previous one.  A coarse row is three
// 16-byte words, copied as such.  Blocks are persistent (one wave, grid-
// stride over the tiles).
#pragma once
#include "compact.cuh"
#include "vfused.cuh"

namespace lcmg {

constexpr int kVcThreads = 256;
constexpr int kVcWR = 2 * kVTile + 2;  // restriction window (fine points of the level) 18 x 18
constexpr int kVcW1 = kVcWR + 4;       // z1 window of the residual's 25-point stencil 22 x 22
constexpr int kVcWF = 2 * kVTile;      // a tile's own fine points 16 x 16
constexpr int kVcW0 = kVcWF + 4;       // z0 window of the sweep's stencil 20 x 20
constexpr int kVcCW = kVTile + 4;      // coarse window of the prolongation onto it 12 x 12

struct VcDownStage {
  uint4 rows[3 * kVcWR * kVcWR];  // K rows on the residual window
  float s[kVcWR * kVcWR];         // their row sums
  float r[kVcW1 * kVcW1];
  float d[kVcW1 * kVcW1];         // D = diag^-1 of the smoother
};
struct VcUpStage {
  uint4 rows[3 * kVcWF * kVcWF];
  float s[kVcWF * kVcWF];
  float r[kVcWF * kVcWF];
  float d[kVcWF * kVcWF];
  float zp[kVcW0 * kVcW0];        // pre-smoothed z1
  float ec[kVcCW * kVcCW];        // coarse correction
};

__device__ __forceinline__ bool vc_inside(const CoarseOpH& op, int i, int j) {
  return i >= 0 && i < op.nv && j >= 0 && j < op.nh;
}

// copies of the element (i, j) of column col of an interleaved vector
__device__ __forceinline__ void vc_copy_vec(float* dst, const float* v, const CoarseOpH& op, int B, int col, int i,
                                            int j) {
  const bool ok = vc_inside(op, i, j);
  cp_async_elem(dst, v + (ok ? ((int64_t)i + (int64_t)j * op.nv) * B + col : 0), v, ok);
}
// the row of point (i, j): three 16-byte words, word w of it
__device__ __forceinline__ void vc_copy_row(uint4* dst, const CoarseOpH& op, int i, int j, int w) {
  const bool ok = vc_inside(op, i, j);
  cp_async16(dst, op.rows + (ok ? 3 * ((int64_t)i + (int64_t)j * op.nv) + w : 0), op.rows, ok);
}

__device__ __forceinline__ void vc_stage_down(VcDownStage& st, const CoarseOpH& op, int B, int col,
                                              const float* __restrict__ dinv, const float* __restrict__ r, int tx,
                                              int ty) {
  const int ri = 2 * kVTile * tx - 1, rj = 2 * kVTile * ty - 1;
  const int oi = ri - 2, oj = rj - 2;
  for (int t = threadIdx.x; t < 3 * kVcWR * kVcWR; t += kVcThreads) {
    const int q = t / 3;
    vc_copy_row(&st.rows[t], op, ri + q % kVcWR, rj + q / kVcWR, t - 3 * q);
  }
  for (int t = threadIdx.x; t < kVcWR * kVcWR; t += kVcThreads) {
    const int i = ri + t % kVcWR, j = rj + t / kVcWR;
    const bool ok = vc_inside(op, i, j);
    cp_async_elem(&st.s[t], op.s + (ok ? (int64_t)i + (int64_t)j * op.nv : 0), op.s, ok);
  }
  for (int t = threadIdx.x; t < kVcW1 * kVcW1; t += kVcThreads) {
    const int i = oi + t % kVcW1, j = oj + t / kVcW1;
    vc_copy_vec(&st.r[t], r, op, B, col, i, j);
    vc_copy_vec(&st.d[t], dinv, op, B, col, i, j);
  }
}

__device__ __forceinline__ void vc_stage_up(VcUpStage& st, const CoarseOpH& op, int B, int col,
                                            const float* __restrict__ dinv, const float* __restrict__ r,
                                            const float* __restrict__ ec, const float* __restrict__ zpre, int tx,
                                            int ty) {
  const int fi = kVcWF * tx, fj = kVcWF * ty;
  for (int t = threadIdx.x; t < 3 * kVcWF * kVcWF; t += kVcThreads) {
    const int q = t / 3;
    vc_copy_row(&st.rows[t], op, fi + q % kVcWF, fj + q / kVcWF, t - 3 * q);
  }
  for (int t = threadIdx.x; t < kVcWF * kVcWF; t += kVcThreads) {
    const int i = fi + t % kVcWF, j = fj + t / kVcWF;
    const bool ok = vc_inside(op, i, j);
    cp_async_elem(&st.s[t], op.s + (ok ? (int64_t)i + (int64_t)j * op.nv : 0), op.s, ok);
    vc_copy_vec(&st.r[t], r, op, B, col, i, j);
    vc_copy_vec(&st.d[t], dinv, op, B, col, i, j);
  }
  for (int t = threadIdx.x; t < kVcW0 * kVcW0; t += kVcThreads)
    vc_copy_vec(&st.zp[t], zpre, op, B, col, fi - 2 + t % kVcW0, fj - 2 + t / kVcW0);
  const int nvc = op.nv / 2, nhc = op.nh / 2;
  const int ci = kVTile * tx - 2, cj = kVTile * ty - 2;
  for (int t = threadIdx.x; t < kVcCW * kVcCW; t += kVcThreads) {
    const int I = ci + t % kVcCW, J = cj + t / kVcCW;
    const bool ok = I >= 0 && I < nvc && J >= 0 && J < nhc;
    cp_async_elem(&st.ec[t], ec + (ok ? ((int64_t)I + (int64_t)J * nvc) * B + col : 0), ec, ok);
  }
}

template <class Stage>
__device__ __forceinline__ Stage* vc_stages() {
  extern __shared__ __align__(16) unsigned char vc_raw[];
  return reinterpret_cast<Stage*>(vc_raw);
}

__global__ void __launch_bounds__(kVcThreads)
    k_vdown_h(CoarseOpH op, int B, const float* __restrict__ dinv, const float* __restrict__ r,
              float* __restrict__ zpre, float* __restrict__ rc, int ntx, int ntiles) {
  VcDownStage* st = vc_stages<VcDownStage>();
  __shared__ float sz1[kVcW1 * kVcW1];
  __shared__ float sres[kVcWR * kVcWR];
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  int buf = 0;
  if ((int)blockIdx.x < ntiles) vc_stage_down(st[0], op, B, col, dinv, r, blockIdx.x % ntx, blockIdx.x / ntx);
  cp_async_commit();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const int next = tile + gridDim.x;
    if (next < ntiles) vc_stage_down(st[buf ^ 1], op, B, col, dinv, r, next % ntx, next / ntx);
    cp_async_commit();
    cp_async_wait_group<1>();  // this tile's copies have landed
    __syncthreads();
    const VcDownStage& S = st[buf];
    const int tx = tile % ntx, ty = tile / ntx;
    const int I0 = kVTile * tx, J0 = kVTile * ty;
    const int ri = 2 * I0 - 1, rj = 2 * J0 - 1;
    // z1 = D r on the window (zero outside the level)
    for (int t = threadIdx.x; t < kVcW1 * kVcW1; t += kVcThreads) sz1[t] = S.d[t] * S.r[t];
    __syncthreads();
    // res = r - K z1 on the restriction window
    for (int t = threadIdx.x; t < kVcWR * kVcWR; t += kVcThreads) {
      const int li = t % kVcWR, lj = t / kVcWR;
      const int i = ri + li, j = rj + lj;
      float v = 0.f;
      if (i >= 0 && i < nv && j >= 0 && j < nh) {
        float k[28];
        op.decode(S.rows[3 * t], S.rows[3 * t + 1], S.rows[3 * t + 2], S.s[t], k);
        const int q = (li + 2) + (lj + 2) * kVcW1;
        auto vz = [&](int di, int dj) { return sz1[q + di + dj * kVcW1]; };
        v = S.r[q] - op.apply_k(k, i, j, vz);
      }
      sres[t] = v;
    }
    // the pre-smoothed z of the tile's own points
    for (int t = threadIdx.x; t < kVcWF * kVcWF; t += kVcThreads) {
      const int li = t % kVcWF, lj = t / kVcWF;
      const int i = 2 * I0 + li, j = 2 * J0 + lj;
      if (i < nv && j < nh) zpre[((int64_t)i + (int64_t)j * nv) * B + col] = sz1[(li + 3) + (lj + 3) * kVcW1];
    }
    __syncthreads();
    // r_c = R res
    for (int t = threadIdx.x; t < kVTile * kVTile; t += kVcThreads) {
      const int I = I0 + t % kVTile, J = J0 + t / kVTile;
      if (I >= nvc || J >= nhc) continue;
      float acc = 0.f;
#pragma unroll
      for (int b = 2 * J - 1; b <= 2 * J + 2; ++b) {
        if (b < 0 || b >= nh) continue;
        const float wb = pw1<float>(b, J, nhc);
#pragma unroll
        for (int a2 = 2 * I - 1; a2 <= 2 * I + 2; ++a2) {
          if (a2 < 0 || a2 >= nv) continue;
          acc += wb * pw1<float>(a2, I, nvc) * sres[(a2 - ri) + (b - rj) * kVcWR];
        }
      }
      rc[((int64_t)I + (int64_t)J * nvc) * B + col] = acc;
    }
    __syncthreads();  // sz1, sres and this stage are rewritten for the tile after next
  }
  cp_async_wait_group<0>();
}

__global__ void __launch_bounds__(kVcThreads)
    k_vup_h(CoarseOpH op, int B, const float* __restrict__ dinv, const float* __restrict__ r,
            const float* __restrict__ ec, const float* __restrict__ zpre, float* __restrict__ zout, int ntx,
            int ntiles, double* __restrict__ part) {
  VcUpStage* st = vc_stages<VcUpStage>();
  __shared__ float s0[kVcW0 * kVcW0];
  __shared__ double sred[kVcThreads / 32];
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  double dacc = 0.0;  // the tiles' r.z, each summed as in k_vup
  int buf = 0;
  if ((int)blockIdx.x < ntiles)
    vc_stage_up(st[0], op, B, col, dinv, r, ec, zpre, blockIdx.x % ntx, blockIdx.x / ntx);
  cp_async_commit();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const int next = tile + gridDim.x;
    if (next < ntiles) vc_stage_up(st[buf ^ 1], op, B, col, dinv, r, ec, zpre, next % ntx, next / ntx);
    cp_async_commit();
    cp_async_wait_group<1>();
    __syncthreads();
    const VcUpStage& S = st[buf];
    const int tx = tile % ntx, ty = tile / ntx;
    const int fi = kVcWF * tx, fj = kVcWF * ty;
    const int oi = fi - 2, oj = fj - 2;
    const int ci = kVTile * tx - 2, cj = kVTile * ty - 2;
    // z0 = z1 + P e_c on the window
    for (int t = threadIdx.x; t < kVcW0 * kVcW0; t += kVcThreads) {
      const int a2 = oi + t % kVcW0, b = oj + t / kVcW0;
      float v = 0.f;
      if (a2 >= 0 && a2 < nv && b >= 0 && b < nh) {
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
            acc += wb * pw1<float>(a2, I, nvc) * S.ec[(I - ci) + (J - cj) * kVcCW];
          }
        }
        v = S.zp[t] + acc;
      }
      s0[t] = v;
    }
    __syncthreads();
    // z = z0 + D (r - K z0) on the tile's own points
    Dot2 dot;
    for (int t = threadIdx.x; t < kVcWF * kVcWF; t += kVcThreads) {
      const int li = t % kVcWF, lj = t / kVcWF;
      const int i = fi + li, j = fj + lj;
      if (i >= nv || j >= nh) continue;
      float k[28];
      op.decode(S.rows[3 * t], S.rows[3 * t + 1], S.rows[3 * t + 2], S.s[t], k);
      const int q = (li + 2) + (lj + 2) * kVcW0;
      auto vz = [&](int di, int dj) { return s0[q + di + dj * kVcW0]; };
      const float kz = op.apply_k(k, i, j, vz);
      const float rv = S.r[t];
      const float zn = s0[q] + S.d[t] * (rv - kz);
      zout[((int64_t)i + (int64_t)j * nv) * B + col] = zn;
      dot.add(rv, zn);
    }
    dacc += dot.value();
    __syncthreads();
  }
  cp_async_wait_group<0>();
  if (part) vblock_sum<kVcThreads>(dacc, sred, part, B, col);
}

}  // namespace lcmg
