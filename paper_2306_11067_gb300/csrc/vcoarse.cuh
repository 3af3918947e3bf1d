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

// Staging: consecutive threads take consecutive elements of the window
// (W and H compile-time, so the row and column of an element cost a
// multiply-shift); entries outside the level are zero-filled.
template <int W, int H>
__device__ __forceinline__ void vc_stage_rows(uint4* dst, const CoarseOpH& op, int i0, int j0) {
  for (int e = threadIdx.x; e < 3 * W * H; e += kVcThreads) {
    const int rr = e / (3 * W), c = e - rr * (3 * W);
    const int i = i0 + c / 3, j = j0 + rr;
    const bool ok = i >= 0 && i < op.nv && j >= 0 && j < op.nh;
    cp_async16(dst + e, op.rows + (ok ? 3 * ((int64_t)i + (int64_t)j * op.nv) + (c - 3 * (c / 3)) : 0), op.rows,
               ok);
  }
}
// a window of one column of an interleaved level vector (nv x nh points)
template <int W, int H>
__device__ __forceinline__ void vc_stage_vec(float* dst, const float* __restrict__ v, int B, int col, int nv, int nh,
                                             int i0, int j0) {
  for (int e = threadIdx.x; e < W * H; e += kVcThreads) {
    const int rr = e / W, c = e - rr * W;
    const int i = i0 + c, j = j0 + rr;
    const bool ok = i >= 0 && i < nv && j >= 0 && j < nh;
    cp_async_elem(dst + e, v + (ok ? ((int64_t)i + (int64_t)j * nv) * B + col : 0), v, ok);
  }
}

__device__ __forceinline__ void vc_stage_down(VcDownStage& st, const CoarseOpH& op, int B, int col,
                                              const float* __restrict__ dinv, const float* __restrict__ r, int tx,
                                              int ty) {
  const int ri = 2 * kVTile * tx - 1, rj = 2 * kVTile * ty - 1;
  vc_stage_rows<kVcWR, kVcWR>(st.rows, op, ri, rj);
  vc_stage_vec<kVcWR, kVcWR>(st.s, op.s, 1, 0, op.nv, op.nh, ri, rj);
  vc_stage_vec<kVcW1, kVcW1>(st.r, r, B, col, op.nv, op.nh, ri - 2, rj - 2);
  vc_stage_vec<kVcW1, kVcW1>(st.d, dinv, B, col, op.nv, op.nh, ri - 2, rj - 2);
}

__device__ __forceinline__ void vc_stage_up(VcUpStage& st, const CoarseOpH& op, int B, int col,
                                            const float* __restrict__ dinv, const float* __restrict__ r,
                                            const float* __restrict__ ec, const float* __restrict__ zpre, int tx,
                                            int ty) {
  const int fi = kVcWF * tx, fj = kVcWF * ty;
  vc_stage_rows<kVcWF, kVcWF>(st.rows, op, fi, fj);
  vc_stage_vec<kVcWF, kVcWF>(st.s, op.s, 1, 0, op.nv, op.nh, fi, fj);
  vc_stage_vec<kVcWF, kVcWF>(st.r, r, B, col, op.nv, op.nh, fi, fj);
  vc_stage_vec<kVcWF, kVcWF>(st.d, dinv, B, col, op.nv, op.nh, fi, fj);
  vc_stage_vec<kVcW0, kVcW0>(st.zp, zpre, B, col, op.nv, op.nh, fi - 2, fj - 2);
  vc_stage_vec<kVcCW, kVcCW>(st.ec, ec, B, col, op.nv / 2, op.nh / 2, kVTile * tx - 2, kVTile * ty - 2);
}

// pw1(a, I) for a = 2I - 1 .. 2I + 2 on a line of nc coarse points
__device__ __forceinline__ void pw1_four(int I, int nc, float (&w)[4]) {
  w[0] = 0.25f;
  w[1] = I == 0 ? 1.f : 0.75f;
  w[2] = I == nc - 1 ? 1.f : 0.75f;
  w[3] = 0.25f;
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
  const float inv_sc = 1.0f / op.sc;  // a power of two
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
    // res = r - K z1 on the restriction window (zero outside the level)
    for (int t = threadIdx.x; t < kVcWR * kVcWR; t += kVcThreads) {
      const int lj = t / kVcWR, li = t - lj * kVcWR;
      const int i = ri + li, j = rj + lj;
      const int q = (li + 2) + (lj + 2) * kVcW1;
      auto vz = [&](int di, int dj) { return sz1[q + di + dj * kVcW1]; };
      const float kz = op.apply_rows(S.rows[3 * t], S.rows[3 * t + 1], S.rows[3 * t + 2], S.s[t], inv_sc, vz);
      sres[t] = (i >= 0 && i < nv && j >= 0 && j < nh) ? S.r[q] - kz : 0.f;
    }
    // the pre-smoothed z of the tile's own points
    for (int t = threadIdx.x; t < kVcWF * kVcWF; t += kVcThreads) {
      const int li = t % kVcWF, lj = t / kVcWF;
      const int i = 2 * I0 + li, j = 2 * J0 + lj;
      if (i < nv && j < nh) zpre[((int64_t)i + (int64_t)j * nv) * B + col] = sz1[(li + 3) + (lj + 3) * kVcW1];
    }
    __syncthreads();
    // r_c = R res (the residual window is zero outside the level, so the
    // terms k_vdown leaves out add nothing)
    for (int t = threadIdx.x; t < kVTile * kVTile; t += kVcThreads) {
      const int I = I0 + t % kVTile, J = J0 + t / kVTile;
      if (I >= nvc || J >= nhc) continue;
      float wa[4], wb[4];
      pw1_four(I, nvc, wa);
      pw1_four(J, nhc, wb);
      const float* rs = sres + (2 * I - 1 - ri) + (2 * J - 1 - rj) * kVcWR;
      float acc = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int m = 0; m < 4; ++m) acc += wb[u] * wa[m] * rs[m + u * kVcWR];
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
  const float inv_sc = 1.0f / op.sc;  // a power of two
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
      const int q = (li + 2) + (lj + 2) * kVcW0;
      auto vz = [&](int di, int dj) { return s0[q + di + dj * kVcW0]; };
      const float kz = op.apply_rows(S.rows[3 * t], S.rows[3 * t + 1], S.rows[3 * t + 2], S.s[t], inv_sc, vz);
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
