// CSR SpMM with the matrix streamed through shared memory.
//
// The operator passes of the normal-equations product (A p, and
// A^T y + lam2 L^T W L p, Sec. 2) read the CSR matrix once and gather the
// vector entries its column indices name.  In the direct kernel (k_spmm) a
// warp loads a row's indices and values and then waits for its gathers, so
// the HBM stream stalls whenever the warps are waiting on L2.  Here the
// rows are cut into chunks (consecutive rows with at most kChunkNnz
// nonzeros and kChunkRows rows) and every block is warp-specialised: one
// producer warp streams the block's chunks into a ring of kStages
// shared-memory stages with bulk asynchronous copies (cp.async.bulk,
// completion counted on a "full" mbarrier per stage), and kConsumerWarps
// consumer warps compute rows from shared memory, each warp releasing a
// stage on its "empty" mbarrier when done.  No block-wide barrier sits in
// the loop, so a warp that finishes its rows moves on to the next chunk.
// A row longer than kChunkNnz is a chunk of its own whose indices and
// values are read from global memory directly.
//
// Every mbarrier wait is bounded (about one second of SM clock); a wait
// that gives up sets *err and the block stops consuming; the producer lets
// the copies it issued land (again bounded) before the block ends.
#pragma once
#include "kernels.cuh"

namespace lcmg {

constexpr int kChunkNnz = 2048;
constexpr int kChunkRows = 32;
constexpr int kStages = 3;
constexpr int kConsumerWarps = 8;
constexpr int kStagedThreads = (kConsumerWarps + 1) * 32;
constexpr long long kWaitCycles = 2000000000LL;

// Byte layout of one stage for matrix values of type V: a header, the row
// pointers rp[ra .. rb), the column indices and values of [ka, kb)
// (ra, ka rounded down and rb, kb up to 16-byte multiples).
template <class V>
struct StageGeo {
  static constexpr int hdr = 0;
  static constexpr int rp = 128;
  static constexpr int rp_bytes = ((kChunkRows + 4) * 8 + 127) / 128 * 128;
  static constexpr int ci = rp + rp_bytes;
  static constexpr int ci_bytes = ((kChunkNnz + 8) * 4 + 127) / 128 * 128;
  static constexpr int va = ci + ci_bytes;
  static constexpr int va_bytes = ((kChunkNnz + 8) * (int)sizeof(V) + 127) / 128 * 128;
  static constexpr int stage = va + va_bytes;
  static constexpr int base = 128;  // 2 x kStages mbarriers first
  static constexpr int total = base + kStages * stage;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// false when the phase has not completed within kWaitCycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// global -> shared bulk copy; bytes a nonzero multiple of 16, both
// addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                          uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct StageHdr {
  int64_t r0, r1, ka, ra;
  int32_t direct;  // 1: the chunk is one long row, read from global memory
};

// Chunk descriptor as read from the chunk table.
struct ChunkDesc {
  int64_t r0, r1, k0, k1;
};
__device__ __forceinline__ ChunkDesc chunk_desc(const SpmmArgs& a, int64_t c) {
  return ChunkDesc{a.ck_row[c], a.ck_row[c + 1], a.ck_nz[c], a.ck_nz[c + 1]};
}

// One chunk into a stage (producer lane only).
template <class V>
__device__ __forceinline__ void stage_issue(const SpmmArgs& a, const V* va, unsigned char* st,
                                            uint64_t* full, const ChunkDesc& d, uint64_t pol) {
  using Geo = StageGeo<V>;
  const int64_t ra = d.r0 & ~1LL, rb = (d.r1 + 2) & ~1LL;  // rp[r0 .. r1] inclusive
  const int direct = (d.k1 - d.k0) > kChunkNnz;
  const int64_t ka = d.k0 & ~3LL, kb = (d.k1 + 3) & ~3LL;
  StageHdr* h = reinterpret_cast<StageHdr*>(st + Geo::hdr);
  h->r0 = d.r0;
  h->r1 = d.r1;
  h->ka = ka;
  h->ra = ra;
  h->direct = direct;
  const uint32_t b_rp = (uint32_t)((rb - ra) * 8);
  // a chunk of empty rows may have nothing to copy (ka == kb): no
  // zero-byte copies are issued
  const uint32_t b_ci = direct ? 0u : (uint32_t)((kb - ka) * 4);
  const uint32_t b_va = direct ? 0u : (uint32_t)((kb - ka) * (int64_t)sizeof(V));
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(full, b_rp + b_ci + b_va);
  bulk_load(st + Geo::rp, a.rp + ra, b_rp, full, pol);
  if (b_ci != 0u) {
    bulk_load(st + Geo::ci, a.ci + ka, b_ci, full, pol);
    bulk_load(st + Geo::va, va + ka, b_va, full, pol);
  }
}

// Same contract and modes as k_spmm (MODE 0: Y = A X; MODE 1: Q = A^T Y +
// lam2 L^T W L P with P.Q partials; MODE 2: ||A X - b||^2 partials; MODE 3:
// R = C - (A^T Y + lam2 L^T W L P) with R.R partials).  Launched with
// kStagedThreads threads and StageGeo<V>::total bytes of dynamic shared
// memory.
template <class V, class T, class TO, int G, int CPG, int MODE>
__global__ void __launch_bounds__(kStagedThreads, (G == 1) ? (sizeof(V) == 4 ? 4 : 2) : 1)
    k_spmm_staged(SpmmArgs a, const V* __restrict__ va, const T* __restrict__ X, TO* __restrict__ Y,
                  FineOp<T> fop, const T* __restrict__ P, const T* __restrict__ C,
                  const double* __restrict__ lam2, const double* __restrict__ bvec,
                  double* __restrict__ part, ScalarFold fold) {
  pdl_entry();
  using Geo = StageGeo<V>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kStages;
  constexpr int S = 32 / G;
  constexpr int U = (G == 1) ? 8 : 4;  // nonzeros per lane in flight
  constexpr bool kPrefetch = (G == 1) && (CPG == 1) && (MODE == 1 || MODE == 3);
  __shared__ double sdot[kConsumerWarps][G * CPG];
  __shared__ volatile int s_abort;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool producer = (warp == kConsumerWarps);
  const int g = lane % G, s = lane / G;
  const int cfirst = a.c0 + blockIdx.y * (G * CPG);
  const int cend = min(a.c0 + a.nb, cfirst + G * CPG);
  const int cbase = cfirst + g * CPG;
  double dacc[CPG];
#pragma unroll
  for (int t = 0; t < CPG; ++t) dacc[t] = 0.0;

  const int64_t first = blockIdx.x, step = gridDim.x;
  const int64_t mine = first < a.nck ? (a.nck - 1 - first) / step + 1 : 0;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int sl = 0; sl < kStages; ++sl) {
      mbar_init(&full[sl], 1);
      mbar_init(&empty[sl], kConsumerWarps);
    }
    mbar_init_fence();
  }
  __syncthreads();

  if (producer) {
    if (lane == 0) {
      const uint64_t pol = l2_evict_first_policy();
      int64_t issued = 0;
      ChunkDesc d = mine > 0 ? chunk_desc(a, first) : ChunkDesc{0, 0, 0, 0};
      for (int64_t i = 0; i < mine; ++i) {
        const int sl = (int)(i % kStages);
        // the stage is free once every consumer warp released its previous use
        if (i >= kStages && !mbar_wait_bounded(&empty[sl], (uint32_t)(((i / kStages) - 1) & 1))) {
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        stage_issue<V>(a, va, smem + Geo::base + sl * Geo::stage, &full[sl], d, pol);
        ++issued;
        if (i + 1 < mine) d = chunk_desc(a, first + (i + 1) * step);  // overlaps the next wait
      }
      if (s_abort) {
        atomicExch(a.err, 1);
        // let the copies in flight land: the last kStages issued chunks
        for (int64_t j = (issued > kStages ? issued - kStages : 0); j < issued; ++j)
          (void)mbar_wait_bounded(&full[j % kStages], (uint32_t)((j / kStages) & 1));
      }
    }
  } else {
    for (int64_t i = 0; i < mine; ++i) {
      const int sl = (int)(i % kStages);
      unsigned char* st = smem + Geo::base + sl * Geo::stage;
      if (!mbar_wait_bounded(&full[sl], (uint32_t)((i / kStages) & 1))) s_abort = 1;
      if (s_abort) break;
      const StageHdr h = *reinterpret_cast<const StageHdr*>(st + Geo::hdr);
      const int64_t* rps = reinterpret_cast<const int64_t*>(st + Geo::rp);
      const int32_t* cis = reinterpret_cast<const int32_t*>(st + Geo::ci);
      const V* vas = reinterpret_cast<const V*>(st + Geo::va);
      for (int64_t r = h.r0 + warp; r < h.r1; r += kConsumerWarps) {
        const int64_t k0 = rps[r - h.ra], k1 = rps[r + 1 - h.ra];
        // one column, A^T pass: lanes 0..9 fetch the epilogue operands of
        // pixel r before the row's gathers so both round trips overlap
        T ep = 0;
        int ii = 0, jj = 0;
        if (MODE == 1 || MODE == 3) {
          jj = (int)(r / fop.nv);
          ii = (int)(r - (int64_t)jj * fop.nv);
        }
        if (kPrefetch && cbase < cend) {
          const int64_t B_ = a.B;
          const int nv = fop.nv;
          switch (lane) {
            case 0: ep = P[r * B_ + cbase]; break;
            case 1: ep = (ii + 1 < nv) ? P[(r + 1) * B_ + cbase] : (T)0; break;
            case 2: ep = (ii > 0) ? P[(r - 1) * B_ + cbase] : (T)0; break;
            case 3: ep = (jj + 1 < fop.nh) ? P[(r + nv) * B_ + cbase] : (T)0; break;
            case 4: ep = (jj > 0) ? P[(r - nv) * B_ + cbase] : (T)0; break;
            case 5: ep = (ii + 1 < nv) ? fop.ws[r] : (T)0; break;
            case 6: ep = (ii > 0) ? fop.ws[r - 1] : (T)0; break;
            case 7: ep = (jj + 1 < fop.nh) ? fop.we[r] : (T)0; break;
            case 8: ep = (jj > 0) ? fop.we[r - nv] : (T)0; break;
            case 9: ep = (MODE == 3) ? C[r * B_ + cbase] : (T)0; break;
            default: break;
          }
        }
        T acc[CPG];
#pragma unroll
        for (int t = 0; t < CPG; ++t) acc[t] = 0;
        for (int64_t kb = k0 + s; kb < k1; kb += S * U) {
          int cu[U];
          T vu[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int64_t k = kb + (int64_t)u * S;
            const bool ok = k < k1;
            if (h.direct) {
              cu[u] = ok ? __ldcs(a.ci + k) : 0;
              vu[u] = ok ? (T)__ldcs(va + k) : (T)0;
            } else {
              cu[u] = ok ? cis[k - h.ka] : 0;
              vu[u] = ok ? (T)vas[k - h.ka] : (T)0;
            }
          }
          T xv[U][CPG];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const T* xr = X + (int64_t)cu[u] * a.B + cbase;
#pragma unroll
            for (int t = 0; t < CPG; ++t) xv[u][t] = (cbase + t < cend) ? xr[t] : (T)0;
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int t = 0; t < CPG; ++t) acc[t] += vu[u] * xv[u][t];
        }
#pragma unroll
        for (int off = G; off < 32; off <<= 1)
#pragma unroll
          for (int t = 0; t < CPG; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], off);
        if (kPrefetch) {
          T o[10];
#pragma unroll
          for (int l = 0; l < 10; ++l) o[l] = __shfl_sync(0xffffffffu, ep, l);
          if (lane == 0 && cbase < cend) {
            const int col = cbase;
            const T pr = o[0];
            // the order of FineOp::lap: +i, -i, +j, -j neighbours
            T lap = 0;
            lap += o[5] * (pr - o[1]);
            lap += o[6] * (pr - o[2]);
            lap += o[7] * (pr - o[3]);
            lap += o[8] * (pr - o[4]);
            const T qv = acc[0] + (T)lam2[col] * lap;
            if (MODE == 1) {
              Y[r * a.B + col] = (TO)qv;
              dacc[0] += to_d(pr) * to_d(qv);
            } else {
              const T rv = o[9] - qv;
              Y[r * a.B + col] = (TO)rv;
              dacc[0] += to_d(rv) * to_d(rv);
            }
          }
        } else if (s == 0) {
#pragma unroll
          for (int t = 0; t < CPG; ++t) {
            const int col = cbase + t;
            if (col >= cend) continue;
            if (MODE == 0) {
              Y[r * a.B + col] = (TO)acc[t];
            } else if (MODE == 1 || MODE == 3) {
              auto pv = [&](int64_t q) { return P[q * a.B + col]; };
              const T lap = fop.lap(r, ii, jj, pv);
              const T qv = acc[t] + (T)lam2[col] * lap;
              if (MODE == 1) {
                Y[r * a.B + col] = (TO)qv;
                dacc[t] += to_d(P[r * a.B + col]) * to_d(qv);
              } else {
                const T rv = C[r * a.B + col] - qv;
                Y[r * a.B + col] = (TO)rv;
                dacc[t] += to_d(rv) * to_d(rv);
              }
            } else {  // MODE 2
              const double e = to_d(acc[t]) - bvec[r * a.nrhs + col / a.nl];
              dacc[t] += e * e;
            }
          }
        }
      }
      // this warp is done with the stage
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sl]);
    }
  }
  __syncthreads();
  if (s_abort) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    return;
  }
  if (MODE != 0) {
    if (!producer && s == 0) {
#pragma unroll
      for (int t = 0; t < CPG; ++t) sdot[warp][g * CPG + t] = dacc[t];
    }
    __syncthreads();
    const int width = cend - cfirst;
    if ((int)threadIdx.x < width) {
      double sum = 0.0;
      for (int w = 0; w < kConsumerWarps; ++w) sum += sdot[w][threadIdx.x];
      part[(int64_t)blockIdx.x * a.B + cfirst + threadIdx.x] = sum;
    }
    if (MODE == 1 && fold.ticket != nullptr) {
      if (last_block(fold.ticket)) fold_alpha(fold.st, a.B, part, (int)gridDim.x);
    }
  }
}

}  // namespace lcmg
