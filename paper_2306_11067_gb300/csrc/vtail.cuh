// The small coarse levels of the V(1,1) cycle (Algorithm 1, nu = 1, FP16
// level operators) and the coarsest-level solve in one kernel.
//
// Below about a thousand points a level's two tile kernels are a few
// microseconds of launch and memory latency each for a few kilobytes of
// work, and a 10-level cycle has several such levels.  Here one block of
// 1024 threads per column runs them all: down the levels (z1 = D r, res = r
// - K z1, r_c = R res), the coarsest solve (the dense inverse of the
// coarsest K(lambda) applied in FP64), and up again (z0 = z1 + P e_c, z =
// z0 + D (r - K z0)), with a block barrier between the steps.  Everything
// the levels read (the FP16 rows, row sums, D and the right-hand side of
// the first of them) is copied into shared memory once, with asynchronous
// copies, and every vector the steps produce stays there: only the
// correction of the first tail level is written back.  At most
// kTailPoints points on the first tail level keep the whole tail within
// about 100 KB of shared memory.  Every point's formulas and the order of
// every sum are those of k_vdown_h, k_vup_h and k_coarse_solve, so the
// cycle is the same operator bit for bit.
#pragma once
#include "compact.cuh"
#include "launch.h"
#include "vfused.cuh"

namespace lcmg {

constexpr int kTailThreads = 1024;
constexpr int kTailMaxLevels = 12;

// one level of the tail and where its arrays live in shared memory (byte
// offsets; the rows 16-byte aligned)
struct TailLevel {
  CoarseOpH op;         // rows and row sums in global memory (copied in)
  const float* dinv;    // global
  const float* rhs;     // global right-hand side (first level only)
  float* z;             // global correction (first level only)
  int o_rows, o_s, o_d, o_r, o_t, o_res, o_z;
};
struct TailArgs {
  int nlev;  // levels in the tail, the last one the coarsest
  TailLevel lv[kTailMaxLevels];
  const double* kinv;  // coarsest inverse, nc x nc per column
  int nc;
};

__global__ void __launch_bounds__(kTailThreads) k_vtail_h(TailArgs a, int B) {
  extern __shared__ __align__(16) unsigned char tail_sm[];
  const int col = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto F = [&](int off) { return reinterpret_cast<float*>(tail_sm + off); };
  // copy in: rows, row sums and D of every level but the coarsest, the
  // right-hand side of the first
  for (int k = 0; k + 1 < a.nlev; ++k) {
    const TailLevel& L = a.lv[k];
    const int n = L.op.nv * L.op.nh;
    uint4* rows = reinterpret_cast<uint4*>(tail_sm + L.o_rows);
    for (int e = threadIdx.x; e < 3 * n; e += kTailThreads) cp_async16(rows + e, L.op.rows + e, L.op.rows, true);
    float* s = F(L.o_s);
    float* d = F(L.o_d);
    for (int p = threadIdx.x; p < n; p += kTailThreads) {
      cp_async_elem(s + p, L.op.s + p, L.op.s, true);
      cp_async_elem(d + p, L.dinv + (int64_t)p * B + col, L.dinv, true);
    }
    if (k == 0) {
      float* r = F(L.o_r);
      for (int p = threadIdx.x; p < n; p += kTailThreads) cp_async_elem(r + p, L.rhs + (int64_t)p * B + col, L.rhs, true);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // down
  for (int k = 0; k + 1 < a.nlev; ++k) {
    const TailLevel& L = a.lv[k];
    const CoarseOpH& op = L.op;
    const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
    const int n = nv * nh;
    const uint4* rows = reinterpret_cast<const uint4*>(tail_sm + L.o_rows);
    const float *s = F(L.o_s), *d = F(L.o_d), *r = F(L.o_r);
    float *t = F(L.o_t), *res = F(L.o_res);
    for (int p = threadIdx.x; p < n; p += kTailThreads) t[p] = d[p] * r[p];
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += kTailThreads) {
      const int j = p / nv, i = p - j * nv;
      float kk[28];
      op.decode(rows[3 * p], rows[3 * p + 1], rows[3 * p + 2], s[p], kk);
      auto vz = [&](int di, int dj) { return t[p + di + dj * nv]; };
      res[p] = r[p] - op.apply_k(kk, i, j, vz);
    }
    __syncthreads();
    float* rc = F(a.lv[k + 1].o_r);
    for (int P = threadIdx.x; P < nvc * nhc; P += kTailThreads) {
      const int J = P / nvc, I = P - J * nvc;
      float acc = 0.f;
#pragma unroll
      for (int b = 2 * J - 1; b <= 2 * J + 2; ++b) {
        if (b < 0 || b >= nh) continue;
        const float wb = pw1<float>(b, J, nhc);
#pragma unroll
        for (int a2 = 2 * I - 1; a2 <= 2 * I + 2; ++a2) {
          if (a2 < 0 || a2 >= nv) continue;
          acc += wb * pw1<float>(a2, I, nvc) * res[a2 + b * nv];
        }
      }
      rc[P] = acc;
    }
    __syncthreads();
  }
  // coarsest: e = K_c^{-1} r_c in FP64, one row per warp (as k_coarse_solve)
  {
    const TailLevel& C = a.lv[a.nlev - 1];
    const float* rc = F(C.o_r);
    float* ec = F(C.o_z);
    const double* M = a.kinv + (int64_t)col * a.nc * a.nc;
    for (int i = warp; i < a.nc; i += kTailThreads / 32) {
      double sum = 0.0;
      for (int q = lane; q < a.nc; q += 32) sum += M[(int64_t)i * a.nc + q] * (double)rc[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
      if (lane == 0) ec[i] = (float)sum;
    }
    __syncthreads();
  }
  // up
  for (int k = a.nlev - 2; k >= 0; --k) {
    const TailLevel& L = a.lv[k];
    const CoarseOpH& op = L.op;
    const int nv = op.nv, nh = op.nh, nvc = nv / 2, nhc = nh / 2;
    const int n = nv * nh;
    const uint4* rows = reinterpret_cast<const uint4*>(tail_sm + L.o_rows);
    const float *s = F(L.o_s), *d = F(L.o_d), *r = F(L.o_r), *t = F(L.o_t);
    const float* ec = F(a.lv[k + 1].o_z);
    float *z0 = F(L.o_res), *z = F(L.o_z);
    for (int p = threadIdx.x; p < n; p += kTailThreads) {
      const int b = p / nv, a2 = p - b * nv;
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
          acc += wb * pw1<float>(a2, I, nvc) * ec[I + J * nvc];
        }
      }
      z0[p] = t[p] + acc;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += kTailThreads) {
      const int j = p / nv, i = p - j * nv;
      float kk[28];
      op.decode(rows[3 * p], rows[3 * p + 1], rows[3 * p + 2], s[p], kk);
      auto vz = [&](int di, int dj) { return z0[p + di + dj * nv]; };
      const float zn = z0[p] + d[p] * (r[p] - op.apply_k(kk, i, j, vz));
      if (k == 0) L.z[(int64_t)p * B + col] = zn;
      else z[p] = zn;
    }
    __syncthreads();
  }
}

}  // namespace lcmg
