// The coarse end of the V-cycle in one launch.
//
// On the small levels of the hierarchy every V-cycle step is a tiny kernel
// whose cost is launch latency.  k_vcycle_tail runs the V-cycle of
// Algorithm 1 on levels k0 .. L-1 (pre-smoothing from zero, residual,
// restriction, the coarsest direct solve, prolongation, post-smoothing) in
// one block of tail_threads<T>() threads (CL = false; steps separated by
// __syncthreads) or in one thread-block cluster of such blocks (CL = true;
// points strided over the whole cluster, steps separated by cluster
// barriers, and data written earlier in the launch read with ld.global.cg
// from L2, so no CTA reads a stale L1 line).  Every thread reaches every
// barrier: no early return, uniform loop bounds.
// Input: the restricted residual of level k0; output: z of level k0.
#pragma once
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace lcmg {

constexpr int kTailMaxLevels = 16;
// threads of a tail block: one CTA, 1024 in FP32 and 512 in FP64, whose
// 25-point stencil rows need more than the 64 registers a 1024-thread block
// allows; in a cluster 512 for both (room for 128 registers, no spills)
template <class T, bool CL = false>
__host__ __device__ constexpr int tail_threads() { return (CL || sizeof(T) == 8) ? 512 : 1024; }

template <class T>
struct TailLevel {
  int nv, nh;
  int64_t n;
  const T* cf;    // coarse coefficient rows (every tail level is a coarse level)
  const T* dinv;  // n x B
  T* rhs;
  T* z;
  T* t;
  T* res;
};

template <class T>
struct TailArgs {
  int B, nl, nu, nc;
  TailLevel<T> lev[kTailMaxLevels];
  const double* kinv;  // coarsest inverse, B x nc x nc
  const T* lam2T;
};

template <class T, bool CL>
__global__ void __launch_bounds__(tail_threads<T, CL>(), 1) k_vcycle_tail(const TailArgs<T> a) {
  pdl_entry();
  namespace cg = cooperative_groups;
  constexpr int kTailThreads = tail_threads<T, CL>();
  const int B = a.B;
  const int rank = CL ? (int)cg::this_cluster().block_rank() : 0;
  const int nctas = CL ? (int)cg::this_cluster().num_blocks() : 1;
  const int tid = rank * kTailThreads + (int)threadIdx.x;  // thread within the launch
  const int nthreads = nctas * kTailThreads;
  const int ppb = nthreads / B;
  const int kk = tid / B;
  const int col = tid - kk * B;
  const bool ok = kk < ppb;
  const T l2 = ok ? a.lam2T[col] : (T)0;
  const int nl = a.nl, nu = a.nu;
  auto sync = [&]() {
    if constexpr (CL) {
      __threadfence();
      cg::this_cluster().sync();
    } else {
      __syncthreads();
    }
  };
  // data written earlier in this launch (rhs below level 0, z, t, res)
  auto ld = [&](const T* q) -> T {
    if constexpr (CL) return __ldcg(q);
    else return *q;
  };

  auto level_loop = [&](const TailLevel<T>& L, auto&& body) {
    if (!ok) return;
    for (int64_t pt = kk; pt < L.n; pt += ppb) {
      const int j = (int)(pt / L.nv), i = (int)(pt - (int64_t)j * L.nv);
      body(pt, i, j);
    }
  };
  auto K_apply = [&](const TailLevel<T>& L, int64_t pt, int i, int j, auto&& v) -> T {
    CoarseOp<T> op{L.nv, L.nh, L.n, L.cf};
    return op.apply(pt, i, j, l2, v);
  };
  auto sweep = [&](const TailLevel<T>& L, const T* zin, T* zout) {
    level_loop(L, [&](int64_t pt, int i, int j) {
      auto v = [&](int64_t q) { return ld(zin + q * B + col); };
      const T kz = K_apply(L, pt, i, j, v);
      zout[pt * B + col] = ld(zin + pt * B + col) + L.dinv[pt * B + col] * (ld(L.rhs + pt * B + col) - kz);
    });
  };

  for (int k = 0; k + 1 < nl; ++k) {
    const TailLevel<T> L = a.lev[k];
    level_loop(L, [&](int64_t pt, int i, int j) {
      const T z1 = L.dinv[pt * B + col] * ld(L.rhs + pt * B + col);
      if (nu < 2) {
        L.z[pt * B + col] = z1;
        return;
      }
      auto v = [&](int64_t q) { return L.dinv[q * B + col] * ld(L.rhs + q * B + col); };
      L.z[pt * B + col] = z1 + L.dinv[pt * B + col] * (ld(L.rhs + pt * B + col) - K_apply(L, pt, i, j, v));
    });
    sync();
    for (int s = 2; s < nu; ++s) {
      sweep(L, L.z, L.t);
      sync();
      level_loop(L, [&](int64_t pt, int, int) { L.z[pt * B + col] = ld(L.t + pt * B + col); });
      sync();
    }
    level_loop(L, [&](int64_t pt, int i, int j) {
      auto v = [&](int64_t q) { return ld(L.z + q * B + col); };
      L.res[pt * B + col] = ld(L.rhs + pt * B + col) - K_apply(L, pt, i, j, v);
    });
    sync();
    const TailLevel<T> C = a.lev[k + 1];
    level_loop(C, [&](int64_t pc, int I, int J) {
      T acc = 0;
      for (int bb = 2 * J - 1; bb <= 2 * J + 2; ++bb) {
        if (bb < 0 || bb >= L.nh) continue;
        const T wb = (T)pw1(bb, J, C.nh);
        for (int aa = 2 * I - 1; aa <= 2 * I + 2; ++aa) {
          if (aa < 0 || aa >= L.nv) continue;
          acc += wb * (T)pw1(aa, I, C.nv) * ld(L.res + ((int64_t)aa + (int64_t)bb * L.nv) * B + col);
        }
      }
      C.rhs[pc * B + col] = acc;
    });
    sync();
  }
  {  // coarsest level
    const TailLevel<T> Lc = a.lev[nl - 1];
    const int nc = a.nc;
    for (int64_t t = tid; t < (int64_t)nc * B; t += nthreads) {
      const int c = (int)(t % B);
      const int i = (int)(t / B);
      const double* M = a.kinv + ((int64_t)c * nc + i) * nc;
      double s = 0.0;
      for (int q = 0; q < nc; ++q) s += M[q] * (double)ld(Lc.rhs + (int64_t)q * B + c);
      Lc.z[(int64_t)i * B + c] = (T)s;
    }
  }
  sync();
  for (int k = nl - 2; k >= 0; --k) {
    const TailLevel<T> L = a.lev[k];
    const TailLevel<T> C = a.lev[k + 1];
    level_loop(L, [&](int64_t pt, int i, int j) {
      const int I0 = i >> 1, J0 = j >> 1;
      const int I1 = (i & 1) ? I0 + 1 : I0 - 1;
      const int J1 = (j & 1) ? J0 + 1 : J0 - 1;
      T acc = 0;
      const int Is[2] = {I0, I1}, Js[2] = {J0, J1};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int J = Js[u];
        if (J < 0 || J >= C.nh) continue;
        const T wb = (T)pw1(j, J, C.nh);
#pragma unroll
        for (int w2 = 0; w2 < 2; ++w2) {
          const int I = Is[w2];
          if (I < 0 || I >= C.nv) continue;
          acc += wb * (T)pw1(i, I, C.nv) * ld(C.z + ((int64_t)I + (int64_t)J * C.nv) * B + col);
        }
      }
      L.z[pt * B + col] = ld(L.z + pt * B + col) + acc;
    });
    sync();
    if (nu % 2 == 1) {
      level_loop(L, [&](int64_t pt, int, int) { L.t[pt * B + col] = ld(L.z + pt * B + col); });
      sync();
    }
    for (int s = 0; s < nu; ++s) {
      if ((nu - s) % 2 == 0) sweep(L, L.z, L.t);
      else sweep(L, L.t, L.z);
      sync();
    }
  }
}

}  // namespace lcmg
