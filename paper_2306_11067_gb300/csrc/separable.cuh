// Separable blur operator.
//
// A blur whose point-spread function is an outer product fv fh^T (a
// Gaussian, or the anisotropic blur of the deblurring example, Sec. 4) is
// the Kronecker product A = A_h (x) A_v of two 1-D zero-boundary Toeplitz
// correlations: A_v acts along the image columns (index i, contiguous in
// memory) and A_h along the rows (index j, stride n_v).  Hence
//
//     A^T A = (A_h^T A_h) (x) (A_v^T A_v) = T_h (x) T_v,
//
// where each T is a symmetric banded matrix of half-bandwidth 2r whose
// interior rows are the autocorrelation t_k = sum_u f_u f_{u+k} and whose
// first and last r rows lose the products that the zero boundary cuts off.
// The normal operator's data term is then two banded 1-D passes of 4r + 1
// taps each (122 multiply-adds per pixel at r = 15, against 2 (2r+1)^2 =
// 1922 for the direct 2-D form), and A, A^T are passes of 2r + 1 taps.
//
// k_band applies one such pass, out(o) = sum_k c_k in(o - H + k) plus the
// per-row corrections of the boundary rows, to every line of the image
// along the contiguous axis (DIR 0) or the strided axis (DIR 1).  A block
// stages a tile of 32 lines x (128 + 2H) samples in shared memory with
// coalesced asynchronous copies; each thread then owns 16 consecutive
// outputs of one line.
// With the tap count TAPS fixed at compile time (the A^T A passes of the
// common radii) the thread streams its 15 + TAPS samples once each from
// shared memory and adds every one into each output it touches, so the
// coefficients are compile-time operands and the window never sits in
// registers; other tap counts run the same sums in chunks of 8 taps
// (TAPS = 0).  DIR 1 is the
// second pass of the normal operator and fuses its epilogue: the
// lam^2 L^T W L p term, the store and the per-block partial sums of p.q
// (or of the true residual, or of ||A x - b||^2).
#pragma once
#include "kernels.cuh"

namespace lcmg {

constexpr int kBandMaxH = 32;                              // taps <= 65
constexpr int kBandChunk = 8;                              // taps per register chunk
constexpr int kBandMaxTaps = 72;                           // 65 rounded up to the chunk
constexpr int kBandSeg = 128;                              // outputs per line per tile
constexpr int kBandLines = 32;                             // lines per tile (one per lane)
constexpr int kBandThreads = 256;
constexpr int kBandR = kBandSeg / (kBandThreads / 32);     // outputs per thread (16)

// One banded 1-D pass: out(o) = sum_{k=0}^{2H} c[k] in(o - H + k) with in
// zero outside the line, plus, for the nlo first and the nhi last outputs
// of the line, sum_k d[row][k] in(o - H + k) (row = o for the first ones,
// nlo + o - (len - nhi) for the last ones).
template <class T>
struct Band {
  int H;
  int nch;             // chunks of kBandChunk taps: ceil((2H + 1) / 8)
  int nlo, nhi;
  const T* d;          // (nlo + nhi) x (2H + 1) corrections, or null
  T c[kBandMaxTaps];   // zero beyond 2H
};

// epilogues of a pass (DIR 1 only, except BAND_STORE)
enum : int {
  BAND_STORE = 0,    // out = v
  BAND_NORMAL = 1,   // q = v + lam2 L^T W L P; out = q; partials of P.q
  BAND_RESID2 = 2,   // partials of (v - b)^2 (no store)
  BAND_TRUERES = 3   // r = C - (v + lam2 L^T W L P); out = r; partials of r.r
};

template <class T>
__host__ __device__ constexpr int band_smem_line(int nch) { return kBandSeg + kBandChunk * nch; }

// shared memory of one block: the staged input tile (line stride LEN + 1)
// and the output tile (line stride kBandSeg + 1)
template <class T>
__host__ __device__ constexpr size_t band_smem_bytes(int nch) {
  return (size_t)kBandLines * ((band_smem_line<T>(nch) + 1) + (kBandSeg + 1)) * sizeof(T);
}

template <class T, class TO, int DIR, int EPI, int TAPS>
__global__ void __launch_bounds__(kBandThreads)
    k_band(int nv, int nh, int B, Band<T> bd, const T* __restrict__ in, TO* __restrict__ out, FineOp<T> fop,
           const T* __restrict__ P, const T* __restrict__ C, const double* __restrict__ lam2,
           const double* __restrict__ bvec, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char band_raw[];
  T* sm = reinterpret_cast<T*>(band_raw);
  __shared__ double sred[kBandThreads / 32];
  const int col = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int len = DIR == 0 ? nv : nh;       // samples along the filter
  const int nlines = DIR == 0 ? nh : nv;
  const int LEN = band_smem_line<T>(bd.nch);
  const int LS = LEN + 1;                   // DIR 0 line stride (odd: no bank conflicts)
  const int nseg = (len + kBandSeg - 1) / kBandSeg;
  const int ntiles = nseg * ((nlines + kBandLines - 1) / kBandLines);
  const int H = bd.H;
  const T l2 = (EPI == BAND_NORMAL || EPI == BAND_TRUERES) ? (T)lam2[col] : (T)0;
  // tile-local index of (line, sample m)
  auto sidx = [&](int line, int m) { return DIR == 0 ? line * LS + m : m * kBandLines + line; };
  auto gpt = [&](int along, int line) -> int64_t {
    return DIR == 0 ? (int64_t)along + (int64_t)line * nv : (int64_t)line + (int64_t)along * nv;
  };
  DotAcc<T> dot;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int seg0 = (tile % nseg) * kBandSeg;
    const int line0 = (tile / nseg) * kBandLines;
    // stage in(seg0 - H + m) for m in [0, LEN) of the tile's lines (zero
    // outside) with asynchronous copies, consecutive threads along the
    // contiguous axis; every copy of the tile is in flight before the wait
    if (DIR == 0) {
      for (int line = w; line < kBandLines; line += kBandThreads / 32) {
        const int ln = line0 + line;
        for (int m = lane; m < LEN; m += 32) {
          const int a = seg0 - H + m;
          const bool ok = a >= 0 && a < len && ln < nlines;
          cp_async_elem(sm + sidx(line, m), in + (ok ? gpt(a, ln) * B + col : 0), in, ok);
        }
      }
    } else {
      for (int e = threadIdx.x; e < kBandLines * LEN; e += kBandThreads) {
        const int ln = line0 + (e & (kBandLines - 1)), m = e / kBandLines;
        const int a = seg0 - H + m;
        const bool ok = a >= 0 && a < len && ln < nlines;
        cp_async_elem(sm + sidx(e & (kBandLines - 1), m), in + (ok ? gpt(a, ln) * B + col : 0), in, ok);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    const int o0 = w * kBandR;  // first output of this thread (tile-local)
    T acc[kBandR];
#pragma unroll
    for (int t = 0; t < kBandR; ++t) acc[t] = 0;
    if constexpr (TAPS > 0) {
      // acc[t] += c[k] in(o0 + t + k): sample m = t + k feeds outputs t with
      // 0 <= m - t < TAPS; every tap term in increasing k, as in the chunked form
      const T* line = sm + sidx(lane, o0);
      constexpr int stride = DIR == 0 ? 1 : kBandLines;
#pragma unroll
      for (int m = 0; m < kBandR + TAPS - 1; ++m) {
        const T v = line[m * stride];
#pragma unroll
        for (int t = 0; t < kBandR; ++t)
          if (m - t >= 0 && m - t < TAPS) acc[t] += bd.c[m - t] * v;
      }
    } else {
      for (int q = 0; q < bd.nch; ++q) {
        T cc[kBandChunk];
#pragma unroll
        for (int k = 0; k < kBandChunk; ++k) cc[k] = bd.c[q * kBandChunk + k];
        T win[kBandR + kBandChunk - 1];
#pragma unroll
        for (int m = 0; m < kBandR + kBandChunk - 1; ++m) win[m] = sm[sidx(lane, o0 + q * kBandChunk + m)];
#pragma unroll
        for (int t = 0; t < kBandR; ++t)
#pragma unroll
          for (int k = 0; k < kBandChunk; ++k) acc[t] += cc[k] * win[t + k];
      }
    }
    // The rows near the ends of the line whose coefficients differ (zero
    // boundary) add sum_k d[row][k] in(o - H + k).  Only the tiles at the
    // ends of a line hold such rows; there every thread of the block takes
    // a share of the (row, line) sums, on the output tile in shared memory
    // (the owners of the first and last outputs alone would hold the block
    // at the barrier for the whole of these sums).
    constexpr int OS = kBandSeg + 1;
    T* so = sm + kBandLines * LS;
    const bool corr = bd.d != nullptr && (seg0 < bd.nlo || seg0 + kBandSeg > len - bd.nhi);  // block-uniform
    if (DIR == 0 || corr) {
#pragma unroll
      for (int t = 0; t < kBandR; ++t) so[lane * OS + o0 + t] = acc[t];
    }
    if (corr) {
      __syncthreads();
      const int taps = 2 * H + 1;
      const int ohi = min(seg0 + kBandSeg, len);
      const int hend = min(ohi, bd.nlo);                             // head rows [seg0, hend)
      const int tbeg = max(seg0, max(len - bd.nhi, bd.nlo));         // tail rows [tbeg, ohi)
      const int nhead = max(0, hend - seg0), nrows = nhead + max(0, ohi - tbeg);
      for (int e = threadIdx.x; e < nrows * kBandLines; e += kBandThreads) {
        const int line = e & (kBandLines - 1), rr = e / kBandLines;
        const int o = rr < nhead ? seg0 + rr : tbeg + (rr - nhead);
        const int row = o < bd.nlo ? o : bd.nlo + o - (len - bd.nhi);
        const T* dr = bd.d + (int64_t)row * taps;
        const int ol = o - seg0;
        T sum = 0;
        for (int k = 0; k < taps; ++k) sum += dr[k] * sm[sidx(line, ol + k)];
        so[line * OS + ol] += sum;
      }
    }
    if constexpr (DIR == 0) {
      // through shared memory, so that the stores run along the contiguous axis
      __syncthreads();
      for (int t = threadIdx.x; t < kBandLines * kBandSeg; t += kBandThreads) {
        const int line = t / kBandSeg, m = t - line * kBandSeg;
        const int a = seg0 + m, ln = line0 + line;
        if (a < len && ln < nlines) out[gpt(a, ln) * B + col] = (TO)so[line * OS + m];
      }
    } else {
      if (corr) {
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kBandR; ++t) acc[t] = so[lane * OS + o0 + t];
      }
      const int i = line0 + lane;
      if (i < nv) {
#pragma unroll
        for (int t = 0; t < kBandR; ++t) {
          const int j = seg0 + o0 + t;
          if (j >= nh) break;
          const int64_t p = (int64_t)i + (int64_t)j * nv;
          if (EPI == BAND_STORE) {
            out[p * B + col] = (TO)acc[t];
          } else if (EPI == BAND_RESID2) {
            const double e = to_d(acc[t]) - bvec[p * B + col];
            dot.add(e, e);
          } else {
            auto pv = [&](int64_t qq) { return P[qq * B + col]; };
            const T kv = acc[t] + l2 * fop.lap(p, i, j, pv);
            if (EPI == BAND_NORMAL) {
              out[p * B + col] = (TO)kv;
              dot.add(P[p * B + col], kv);
            } else {
              const T rv = C[p * B + col] - kv;
              out[p * B + col] = (TO)rv;
              dot.add(rv, rv);
            }
          }
        }
      }
    }
    __syncthreads();  // the tile buffer is reloaded by the next tile
  }
  if (EPI != BAND_STORE) {
    double dacc = dot.value();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, off);
    if (lane == 0) sred[w] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < kBandThreads / 32; ++k) s += sred[k];
      part[(int64_t)blockIdx.x * B + col] = s;
    }
  }
}

// diag(A^T A)_p = T_v[i][i] T_h[j][j]
static __global__ void k_sep_diag(int nv, int nh, const double* __restrict__ dv, const double* __restrict__ dh,
                                  double* __restrict__ diag) {
  const int64_t n = (int64_t)nv * nh;
  for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n; p += (int64_t)gridDim.x * kBlock) {
    const int j = (int)(p / nv), i = (int)(p - (int64_t)j * nv);
    diag[p] = dv[i] * dh[j];
  }
}

}  // namespace lcmg
