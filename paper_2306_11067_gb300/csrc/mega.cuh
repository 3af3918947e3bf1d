// One PCG iteration's work between the two operator passes, in a single
// launch on one thread-block cluster:
//
//   alpha = rz / p^T q;  x += alpha p;  r -= alpha q;  ||r||^2
//   z = B(lambda) r      (the whole V-cycle of Algorithm 1: pre-smoothing,
//                         residual, restriction, coarsest solve,
//                         prolongation, post-smoothing on every level)
//   r^T z, beta, convergence;  p = z + beta p
//
// Steps are separated by cluster barriers (hardware barrier.cluster; every
// thread of every CTA reaches every barrier: there is no early return and
// every loop bound is uniform).  The barrier's release/acquire semantics
// order every global write before it with every read after it across the
// cluster; the CG variant additionally reads such data with ld.global.cg
// (from L2, bypassing L1).
#pragma once
#include <cooperative_groups.h>

#include "kernels.cuh"
#include "mega_launch.h"

namespace lcmg {

constexpr int kMegaThreads = 512;
constexpr int kMaxLevels = kMegaMaxLevels;
constexpr int kMaxClusterCtas = kMegaMaxCtas;

template <class T>
struct MegaLevel {
  int nv, nh;
  int64_t n;
  int fine;
  const T* ws;    // fine level
  const T* we;
  const T* ga;
  const T* cf;    // coarse levels
  const T* dinv;  // n x B
  T* rhs;         // level 0: the PCG residual r
  T* z;           // level 0: the PCG z
  T* t;
  T* res;
};

template <class T>
struct MegaArgs {
  int B, nlev, nu, nc;
  MegaLevel<T> lev[kMaxLevels];
  const double* kinv;   // coarsest inverse, B x nc x nc
  T* x;                 // FP64 path: x; mixed path: the FP32 increment since the last update
  T* p;
  const T* q;
  const T* lam2T;
  ColState st;
  const double* pq_part;
  int nblk_pq;
  double* cta_part;     // [kMaxClusterCtas][2][B]
  int maxit;
  double rel_trigger;
};

// Loads of data written earlier in the same launch by other CTAs: plain
// loads (ordered by the cluster barrier's release/acquire semantics) or,
// with CG, ld.global.cg straight from L2.
template <bool CG, class T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

__device__ __forceinline__ void cluster_barrier() {
  __threadfence();
  cooperative_groups::this_cluster().sync();
}

template <class T, bool CG>
__global__ void __launch_bounds__(kMegaThreads, 1) k_pcg_mega(const MegaArgs<T> a) {
  namespace cg = cooperative_groups;
  __shared__ double s_alpha[kMaxB];
  __shared__ int s_act[kMaxB];
  __shared__ double s_red[kMegaThreads];
  __shared__ double s_beta[kMaxB];
  __shared__ int s_go[kMaxB];
  __shared__ int s_vote[kMaxB];
  // per-column state as it was at kernel entry: CTA 0 rewrites the global
  // copies in the last step while other CTAs may still be reading
  __shared__ double s_rz[kMaxB], s_tol2cc[kMaxB], s_rmax[kMaxB];
  __shared__ int s_iters[kMaxB];
  __shared__ int s_act0[kMaxB], s_stt0[kMaxB];

  const int rank = (int)cg::this_cluster().block_rank();
  const int nctas = (int)cg::this_cluster().num_blocks();
  const int B = a.B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // cluster-wide (point, column) mapping
  const int gt = rank * kMegaThreads + threadIdx.x;
  const int ppb = (nctas * kMegaThreads) / B;
  const int kk = gt / B;
  const int col = gt - kk * B;
  const bool ok = kk < ppb;
  const ColState st = a.st;

  // CTA partial of a per-thread value for every column, in a fixed order
  // (the threads of this CTA that own column c are t = t0(c) + B m), written
  // to cta_part[rank][slot][c].  Called by all threads of the CTA.
  auto cta_column_sums = [&](double v, int slot) {
    s_red[threadIdx.x] = ok ? v : 0.0;
    __syncthreads();
    if ((int)threadIdx.x < B) {
      const int c = threadIdx.x;
      const int t0 = ((c - (rank * kMegaThreads) % B) % B + B) % B;
      double s = 0.0;
      for (int t = t0; t < kMegaThreads; t += B) s += s_red[t];
      a.cta_part[(rank * 2 + slot) * B + c] = s;
    }
    __syncthreads();
  };

  // ---- S0: alpha per column (every CTA computes the same values) -------
  for (int c = warp; c < B; c += kMegaThreads / 32) {
    const int act = st.active[c];
    double pq = 0.0;
    if (act) {
      for (int b = lane; b < a.nblk_pq; b += 32) pq += a.pq_part[(int64_t)b * B + c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) pq += __shfl_xor_sync(0xffffffffu, pq, off);
    }
    if (lane == 0) {
      // no global state is written before the last step, so every CTA
      // reads the same entry values here
      int go = act;
      double al = 0.0;
      int stt = -1;
      const double rz_old = st.rz[c];
      if (act) {
        if (!isfinite(pq)) { go = 0; stt = ST_NONFINITE; }
        else if (!(pq > 0.0)) { go = 0; stt = ST_BREAKDOWN; }
        else al = rz_old / pq;
      }
      s_alpha[c] = al;
      s_act0[c] = act;
      s_act[c] = go;
      s_stt0[c] = stt;
      s_rz[c] = rz_old;
      s_tol2cc[c] = st.tol2cc[c];
      s_rmax[c] = st.rmax[c];
      s_iters[c] = st.iters[c] + act;
    }
  }
  __syncthreads();

  // ---- S1: x += alpha p ; r -= alpha q ; ||r||^2 ------------------------
  const MegaLevel<T> L0 = a.lev[0];
  {
    double rr = 0.0;
    if (ok && s_act[col]) {
      const T al = (T)s_alpha[col];
      for (int64_t i = kk; i < L0.n; i += ppb) {
        const int64_t e = i * B + col;
        a.x[e] = a.x[e] + al * a.p[e];
        const T rn = L0.rhs[e] - al * a.q[e];
        L0.rhs[e] = rn;
        rr += (double)rn * (double)rn;
      }
    }
    cta_column_sums(rr, 0);
  }
  cluster_barrier();

  // ---- V-cycle ----------------------------------------------------------
  auto level_loop = [&](const MegaLevel<T>& L, auto&& body) {
    if (!ok) return;
    for (int64_t pt = kk; pt < L.n; pt += ppb) {
      const int j = (int)(pt / L.nv), i = (int)(pt - (int64_t)j * L.nv);
      body(pt, i, j);
    }
  };
  const T l2 = ok ? a.lam2T[col] : (T)0;

  auto K_apply = [&](const MegaLevel<T>& L, int64_t pt, int i, int j, auto&& v) -> T {
    if (L.fine) {
      FineOp<T> op{L.nv, L.nh, L.ws, L.we, L.ga};
      return op.apply(pt, i, j, l2, v);
    }
    CoarseOp<T> op{L.nv, L.nh, L.n, L.cf};
    return op.apply(pt, i, j, l2, v);
  };

  // one sweep zout = zin + dinv (rhs - K zin); optionally the r.z partial
  auto sweep = [&](const MegaLevel<T>& L, const T* zin, T* zout, double* dot) {
    level_loop(L, [&](int64_t pt, int i, int j) {
      auto v = [&](int64_t qq) { return ldv<CG>(zin + qq * B + col); };
      const T kz = K_apply(L, pt, i, j, v);
      const T rv = ldv<CG>(L.rhs + pt * B + col);
      const T zn = ldv<CG>(zin + pt * B + col) + L.dinv[pt * B + col] * (rv - kz);
      zout[pt * B + col] = zn;
      if (dot) *dot += (double)rv * (double)zn;
    });
  };

  const int nl = a.nlev;
  const int nu = a.nu;
  for (int k = 0; k + 1 < nl; ++k) {
    const MegaLevel<T> L = a.lev[k];
    // pre-smoothing from zero: z1 = dinv rhs ; z2 = z1 + dinv (rhs - K z1)
    level_loop(L, [&](int64_t pt, int i, int j) {
      const T z1 = L.dinv[pt * B + col] * ldv<CG>(L.rhs + pt * B + col);
      if (nu < 2) {
        L.z[pt * B + col] = z1;
        return;
      }
      auto v = [&](int64_t qq) { return L.dinv[qq * B + col] * ldv<CG>(L.rhs + qq * B + col); };
      const T kz = K_apply(L, pt, i, j, v);
      L.z[pt * B + col] = z1 + L.dinv[pt * B + col] * (ldv<CG>(L.rhs + pt * B + col) - kz);
    });
    cluster_barrier();
    for (int s = 2; s < nu; ++s) {  // remaining pre-sweeps, ping-pong through t
      sweep(L, L.z, L.t, nullptr);
      cluster_barrier();
      level_loop(L, [&](int64_t pt, int, int) { L.z[pt * B + col] = ldv<CG>(L.t + pt * B + col); });
      cluster_barrier();
    }
    // residual
    level_loop(L, [&](int64_t pt, int i, int j) {
      auto v = [&](int64_t qq) { return ldv<CG>(L.z + qq * B + col); };
      L.res[pt * B + col] = ldv<CG>(L.rhs + pt * B + col) - K_apply(L, pt, i, j, v);
    });
    cluster_barrier();
    // restriction rhs_{k+1} = P^T res_k
    const MegaLevel<T> C = a.lev[k + 1];
    level_loop(C, [&](int64_t pc, int I, int J) {
      T acc = 0;
      for (int bb = 2 * J - 1; bb <= 2 * J + 2; ++bb) {
        if (bb < 0 || bb >= L.nh) continue;
        const T wb = (T)pw1(bb, J, C.nh);
        for (int aa = 2 * I - 1; aa <= 2 * I + 2; ++aa) {
          if (aa < 0 || aa >= L.nv) continue;
          acc += wb * (T)pw1(aa, I, C.nv) * ldv<CG>(L.res + ((int64_t)aa + (int64_t)bb * L.nv) * B + col);
        }
      }
      C.rhs[pc * B + col] = acc;
    });
    cluster_barrier();
  }
  // coarsest level: z = K_c^{-1} rhs (FP64), one thread per (row, column);
  // the thread's column is gt mod B, as in every other step
  double rz1 = 0.0;
  {
    const MegaLevel<T> Lc = a.lev[nl - 1];
    const int nc = a.nc;
    for (int64_t t = gt; t < (int64_t)nc * B; t += (int64_t)nctas * kMegaThreads) {
      const int c = (int)(t % B);
      const int i = (int)(t / B);
      const double* M = a.kinv + ((int64_t)c * nc + i) * nc;
      double s = 0.0;
      for (int q = 0; q < nc; ++q) s += M[q] * (double)ldv<CG>(Lc.rhs + (int64_t)q * B + c);
      Lc.z[(int64_t)i * B + c] = (T)s;
      if (nl == 1) rz1 += (double)ldv<CG>(Lc.rhs + (int64_t)i * B + c) * (double)(T)s;  // one level: r.z here
    }
  }
  cluster_barrier();
  double rz = rz1;
  for (int k = nl - 2; k >= 0; --k) {
    const MegaLevel<T> L = a.lev[k];
    const MegaLevel<T> C = a.lev[k + 1];
    // z_k += P z_{k+1}
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
          acc += wb * (T)pw1(i, I, C.nv) * ldv<CG>(C.z + ((int64_t)I + (int64_t)J * C.nv) * B + col);
        }
      }
      L.z[pt * B + col] = ldv<CG>(L.z + pt * B + col) + acc;
    });
    cluster_barrier();
    // post-smoothing, nu sweeps ending in z (ping-pong through t; with an
    // odd count the iterate is first copied into t); the last sweep at
    // level 0 adds the r.z partials
    if (nu % 2 == 1) {
      level_loop(L, [&](int64_t pt, int, int) { L.t[pt * B + col] = ldv<CG>(L.z + pt * B + col); });
      cluster_barrier();
    }
    for (int s = 0; s < nu; ++s) {
      const bool last = (s == nu - 1);
      const bool into_t = ((nu - s) % 2 == 0);  // an even number left: write t
      double* dot = (k == 0 && last) ? &rz : nullptr;
      if (into_t) sweep(L, L.z, L.t, dot);
      else sweep(L, L.t, L.z, dot);
      cluster_barrier();
    }
  }
  cta_column_sums(rz, 1);
  cluster_barrier();

  // ---- beta, convergence, p = z + beta p --------------------------------
  if ((int)threadIdx.x < B) {
    const int c = threadIdx.x;
    double rr = 0.0, rzn = 0.0;
    for (int r2 = 0; r2 < nctas; ++r2) {
      rr += a.cta_part[(r2 * 2 + 0) * B + c];
      rzn += a.cta_part[(r2 * 2 + 1) * B + c];
    }
    int go = s_act[c];
    double be = 0.0;
    int stt = -1, pend = 0, vote = 0;
    if (go) {
      if (!isfinite(rr) || !isfinite(rzn)) { go = 0; stt = ST_NONFINITE; }
      else if (rr <= s_tol2cc[c]) { go = 0; pend = 1; }
      else if (s_iters[c] >= a.maxit) { go = 0; stt = ST_MAXIT; }
      else if (!(rzn > 0.0)) { go = 0; stt = ST_BREAKDOWN; }
      else {
        be = rzn / s_rz[c];
        vote = (a.rel_trigger > 0.0 && rr < a.rel_trigger * s_rmax[c]) ? 1 : 0;
      }
    }
    s_beta[c] = be;
    s_go[c] = go;
    s_vote[c] = vote;
    if (rank == 0 && s_act0[c]) {
      // all state writes of the iteration happen here, by CTA 0 only
      st.iters[c] = s_iters[c];
      st.alpha[c] = s_alpha[c];
      if (s_stt0[c] >= 0) {
        st.status[c] = s_stt0[c];
        st.active[c] = 0;
      } else {
        st.rr[c] = rr;
        st.beta[c] = be;
        if (go) st.rz[c] = st.rz2[c] = rzn;
        if (!go) st.active[c] = 0;
        if (stt >= 0) st.status[c] = stt;
        if (pend) st.pending[c] = 1;
      }
    }
  }
  __syncthreads();
  if (rank == 0 && threadIdx.x == 0) {
    // counts from this CTA's own decisions (the globals it just wrote)
    int na = 0, np = 0, nvote = 0;
    for (int c = 0; c < B; ++c) {
      na += s_go[c];
      np += st.pending[c];
      nvote += s_vote[c];
    }
    st.counters[0] = na;
    st.counters[1] = np;
    st.counters[2] = nvote;
  }
  if (ok && s_go[col]) {
    const T be = (T)s_beta[col];
    for (int64_t i = kk; i < L0.n; i += ppb) {
      const int64_t e = i * B + col;
      a.p[e] = L0.z[e] + be * a.p[e];
    }
  }
}

}  // namespace lcmg
