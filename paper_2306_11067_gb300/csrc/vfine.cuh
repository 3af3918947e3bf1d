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


// ---------------------------------------------------------------------------
// Row-streaming forms of the two FP16 kernels (the default).  A warp owns
// 32 consecutive points along i (one per lane) and walks down a strip of
// rows j: the neighbours along j of the point a lane is at are values it
// computed one row earlier or one row ahead (kept in registers), those
// along i are the neighbouring lanes' values (warp shuffles).  The two edge
// lanes of a warp compute only what their neighbours need (the halo), so a
// warp produces 30 points of z (k_vfine_up_s) or 14 coarse points of r_c
// (k_vfine_down_s) per row; a strip is at most kStripRows rows (kStripCoarse
// coarse rows), fewer on small grids, so that the strips fill the GPU.  No
// shared memory, no barrier; a row's loads
// are issued one row ahead of their use, from addresses clamped into the
// arrays, and every per-point step is branch-free (selects), so that a
// lane's work per row is its arithmetic and little else.
//
// Each point's formulas are those of k_vfine_up / k_vfine_down, with two
// changes of rounding: D^{-1} = 1 / (2 lam^2 sum w + g) (or omega / (lam^2
// sum w + g)) is taken with the fast division (__fdividef, within 2 ulp),
// the same value in both kernels, so the cycle stays one fixed symmetric
// operator; and r_c = P^T res is summed per fine row along i first, then
// along j.  32-bit indices: the launcher takes this path while
// n_v n_h B < 2^31.
// ---------------------------------------------------------------------------
constexpr int kStripRows = 32;    // most fine rows of z per k_vfine_up_s strip
constexpr int kStripCoarse = 16;  // most coarse rows of r_c per k_vfine_down_s strip
constexpr int kUpCols = 30;       // z columns per warp
constexpr int kDownCols = 14;     // r_c columns per warp

// the raw data of the lane's point p = i + j n_v of one row: FP16 w_s(p),
// w_s(p - 1), w_e(p), diag(A^T A)(p), r(p) and, for the up kernel, the four
// coarse corrections of P e_c (element stride S of the interleaved vectors)
struct RawRow {
  __half s, n, e, g;
  float r;
  float c[4];
};
template <bool kCoarse>
__device__ __forceinline__ RawRow fine_load(const __half* __restrict__ ws, const __half* __restrict__ we,
                                            const __half* __restrict__ ga, const float* __restrict__ r,
                                            const float* __restrict__ ec, int S, int col, bool in, int p, int ea,
                                            int eb, int Iac, int Ibc) {
  RawRow q;
  const int pc = in ? p : 0;
  q.s = ws[pc];
  q.n = ws[pc > 0 ? pc - 1 : 0];
  q.e = we[pc];
  q.g = ga[pc];
  q.r = r[pc * S + col];
  if (kCoarse) {
    q.c[0] = ec[(ea + Iac) * S + col];
    q.c[1] = ec[(ea + Ibc) * S + col];
    q.c[2] = ec[(eb + Iac) * S + col];
    q.c[3] = ec[(eb + Ibc) * S + col];
  }
  return q;
}

// the point data a lane carries from one row to the next
struct FineRow {
  float z;     // z1 = D^{-1} r (down) or z0 = z1 + P e_c (up)
  float r, d;  // r and D^{-1}
  float s, n, e, w, g;
};

// weights, D^{-1} and z1 of the lane's point (all zero outside the grid);
// w_prev = e of (i, j - 1)
__device__ __forceinline__ FineRow fine_row(const RawRow& q, float sw, float sg, float l2, int smoother, float omega,
                                            bool in, bool has_s, bool has_n, bool has_e, float w_prev) {
  FineRow f;
  f.s = (in && has_s) ? __half2float(q.s) * sw : 0.f;
  f.n = (in && has_n) ? __half2float(q.n) * sw : 0.f;
  f.e = (in && has_e) ? __half2float(q.e) * sw : 0.f;
  f.w = w_prev;
  f.g = in ? __half2float(q.g) * sg : 0.f;
  f.r = in ? q.r : 0.f;
  const float sum = f.s + f.n + f.e + f.w;
  const float dv = smoother == 0 ? __fdividef(1.0f, 2.0f * l2 * sum + f.g) : __fdividef(omega, l2 * sum + f.g);
  f.d = in ? dv : 0.f;
  f.z = f.d * f.r;
  return f;
}

// (K z)_p from the lane's row record and its neighbours' z
__device__ __forceinline__ float fine_row_kz(const FineRow& f, float l2, float zs, float zn, float ze, float zw) {
  const float zp = f.z;
  const float acc = f.s * (zp - zs) + f.n * (zp - zn) + f.e * (zp - ze) + f.w * (zp - zw);
  return l2 * acc + f.g * zp;
}

// pw1 of the two coarse neighbours of fine index a on a line of n = 2 nc
// points: the nearer one (3/4, or 1 at the ends of the line) and the other
// one (1/4, or 0 at the ends, where it falls outside)
__device__ __forceinline__ void pw1_pair(int a, int n, float& wnear, float& wfar) {
  const bool edge = a == 0 || a == n - 1;
  wnear = edge ? 1.f : 0.75f;
  wfar = edge ? 0.f : 0.25f;
}

template <bool kUnit>
__global__ void __launch_bounds__(kFineThreads)
    k_vfine_up_s(FineOpH op, int B, const float* __restrict__ lam2, int smoother, float omega,
                 const float* __restrict__ r, const float* __restrict__ ec, float* __restrict__ zout, int nsi,
                 int nstrips, int rows, double* __restrict__ part) {
  __shared__ double sred[kFineThreads / 32];
  const unsigned FULL = 0xffffffffu;
  const int S = kUnit ? 1 : B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  const __half* __restrict__ ws = op.ws;
  const __half* __restrict__ we = op.we;
  const __half* __restrict__ ga = op.ga;
  const float sw = op.sw, sg = op.sg;
  const float l2 = lam2[col];
  Dot2 dot;
  for (int st = blockIdx.x * (kFineThreads / 32) + warp; st < nstrips; st += gridDim.x * (kFineThreads / 32)) {
    const int i = (st % nsi) * kUpCols - 1 + lane;
    const int j0 = (st / nsi) * rows, j1 = min(j0 + rows, nh);
    const bool in_i = i >= 0 && i < nv, has_s = i + 1 < nv, has_n = i > 0;
    const bool out = lane >= 1 && lane <= kUpCols && i < nv;
    // interpolation along i (fixed for the lane): coarse columns Ia, Ib
    const int Ia = i >> 1;
    float waA, waB;
    pw1_pair(i, nv, waA, waB);
    const int Iac = min(max(Ia, 0), nvc - 1);
    const int Ibc = min(max((i & 1) ? Ia + 1 : Ia - 1, 0), nvc - 1);
    auto load = [&](int j, int q) {
      const int Ja = min(max(j >> 1, 0), nhc - 1);
      const int Jb = min(max((j & 1) ? Ja + 1 : Ja - 1, 0), nhc - 1);
      return fine_load<true>(ws, we, ga, r, ec, S, col, in_i && j >= 0 && j < nh, q, Ja * nvc, Jb * nvc, Iac, Ibc);
    };
    // z0 = D^{-1} r + P e_c at row j (zero outside the grid)
    auto row = [&](const RawRow& q, int j, float w_prev) {
      const bool in = in_i && j >= 0 && j < nh;
      FineRow f = fine_row(q, sw, sg, l2, smoother, omega, in, has_s, has_n, j + 1 < nh, w_prev);
      float wbA, wbB;
      pw1_pair(j, nh, wbA, wbB);
      float acc = 0.f;  // the terms in the order of k_vfine_up (a zero weight adds nothing)
      acc += wbA * waA * q.c[0];
      acc += wbA * waB * q.c[1];
      acc += wbB * waA * q.c[2];
      acc += wbB * waB * q.c[3];
      f.z += in ? acc : 0.f;
      return f;
    };
    int p = i + (j0 - 1) * nv;  // the lane's point in row j0 - 1
    float we_prev = 0.f;        // e of the row above, the w of the next row
    if (j0 - 2 >= 0 && in_i && j0 - 1 < nh) we_prev = __half2float(we[p - nv]) * sw;
    RawRow qn = load(j0 + 1, p + 2 * nv);  // in flight while rows j0 - 1 and j0 are finished
    FineRow fm = row(load(j0 - 1, p), j0 - 1, we_prev);
    p += nv;
    FineRow fc = row(load(j0, p), j0, fm.e);
    for (int j = j0; j < j1; ++j) {
      const RawRow qj = qn;
      qn = load(j + 2, p + 2 * nv);  // the loads of the row after next
      const FineRow fp = row(qj, j + 1, fc.e);
      const float zs = __shfl_down_sync(FULL, fc.z, 1);
      const float zn = __shfl_up_sync(FULL, fc.z, 1);
      const float zn1 = fc.z + fc.d * (fc.r - fine_row_kz(fc, l2, zs, zn, fp.z, fm.z));
      if (out) zout[p * S + col] = zn1;
      dot.add(out ? fc.r : 0.f, out ? zn1 : 0.f);
      fm = fc;
      fc = fp;
      p += nv;
    }
  }
  if (part) {
    double dacc = dot.value();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dacc += __shfl_xor_sync(FULL, dacc, off);
    if (lane == 0) sred[warp] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int k = 0; k < kFineThreads / 32; ++k) sum += sred[k];
      part[(int64_t)blockIdx.x * B + col] = sum;
    }
  }
}

template <bool kUnit>
__global__ void __launch_bounds__(kFineThreads)
    k_vfine_down_s(FineOpH op, int B, const float* __restrict__ lam2, int smoother, float omega,
                   const float* __restrict__ r, float* __restrict__ rc, int nsi, int nstrips, int crows) {
  const unsigned FULL = 0xffffffffu;
  const int S = kUnit ? 1 : B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y;
  const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
  const __half* __restrict__ ws = op.ws;
  const __half* __restrict__ we = op.we;
  const __half* __restrict__ ga = op.ga;
  const float sw = op.sw, sg = op.sg;
  const float l2 = lam2[col];
  for (int st = blockIdx.x * (kFineThreads / 32) + warp; st < nstrips; st += gridDim.x * (kFineThreads / 32)) {
    const int I0 = (st % nsi) * kDownCols, J0 = (st / nsi) * crows;
    const int i = 2 * I0 - 2 + lane;  // z1 at every lane, res at lanes 1..30
    const bool in_i = i >= 0 && i < nv, has_s = i + 1 < nv, has_n = i > 0;
    // restriction along i: coarse column I = I0 + lane (lanes < 14) from the
    // residual at fine columns 2I - 1 .. 2I + 2 (lanes 2 lane + 1 .. 2 lane + 4)
    const int I = I0 + lane;
    const bool out = lane < kDownCols && I < nvc;
    float wa[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int a2 = 2 * I - 1 + m;
      wa[m] = (a2 >= 0 && a2 < nv && I < nvc) ? pw1<float>(a2, I, nvc) : 0.f;
    }
    const int jb0 = 2 * J0 - 1, jb1 = min(2 * (J0 + crows), nh);  // residual rows [jb0, jb1]
    int p = i + (jb0 - 1) * nv;  // the lane's point in row jb0 - 1
    float we_prev = 0.f;
    if (jb0 - 2 >= 0 && in_i && jb0 - 1 < nh) we_prev = __half2float(we[p - nv]) * sw;
    auto load = [&](int j, int q) {
      return fine_load<false>(ws, we, ga, r, nullptr, S, col, in_i && j >= 0 && j < nh, q, 0, 0, 0, 0);
    };
    auto row = [&](const RawRow& q, int j, float w_prev) {
      return fine_row(q, sw, sg, l2, smoother, omega, in_i && j >= 0 && j < nh, has_s, has_n, j + 1 < nh, w_prev);
    };
    RawRow qn = load(jb0 + 1, p + 2 * nv);  // in flight while rows jb0 - 1 and jb0 are finished
    FineRow fm = row(load(jb0 - 1, p), jb0 - 1, we_prev);
    p += nv;
    FineRow fc = row(load(jb0, p), jb0, fm.e);
    float prev = 0.f, cur = 0.f;  // r_c of coarse rows (b - 1) / 2 and (b + 1) / 2 being summed
    for (int b = jb0; b <= jb1; ++b) {
      const RawRow qb = qn;
      qn = load(b + 2, p + 2 * nv);  // the loads of the row after next
      const FineRow fp = row(qb, b + 1, fc.e);
      const float zs = __shfl_down_sync(FULL, fc.z, 1);
      const float zn = __shfl_up_sync(FULL, fc.z, 1);
      // res = r - K z1, zero outside the grid (so that it adds nothing below)
      const bool in = in_i && b >= 0 && b < nh;
      const float res = in ? fc.r - fine_row_kz(fc, l2, zs, zn, fp.z, fm.z) : 0.f;
      float ti = 0.f;  // sum over a of pw1(a, I) res(a, b)
#pragma unroll
      for (int m = 0; m < 4; ++m) ti += wa[m] * __shfl_sync(FULL, res, (2 * lane + 1 + m) & 31);
      const float wb = (b == 0 || b == nh - 1) ? 1.f : 0.75f;  // pw1(b, b / 2)
      const int m = b >> 1;
      if ((b & 1) == 0) {  // b = 2m: the last term of coarse row m - 1, the second of row m
        prev += 0.25f * ti;
        if (out && m - 1 >= J0 && m - 1 < nhc) rc[(I + (m - 1) * nvc) * S + col] = prev;
        prev = cur + wb * ti;
        cur = 0.f;
      } else {  // b = 2m + 1: the third term of row m, the first of row m + 1
        prev += wb * ti;
        cur += 0.25f * ti;
      }
      fm = fc;
      fc = fp;
      p += nv;
    }
  }
}

}  // namespace lcmg
