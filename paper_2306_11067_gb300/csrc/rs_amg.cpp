// Classical AMG setup on the host (Sec. 3.1); declarations and the rules in
// rs_amg.h.
#include "rs_amg.h"

#include <algorithm>
#include <functional>
#include <queue>
#include <thread>
#include <utility>

namespace lcmg {
namespace amg {

static double entry(const HostCsr& K, int64_t row, int32_t col) {
  const int32_t* b = K.ci.data() + K.rp[row];
  const int32_t* e = K.ci.data() + K.rp[row + 1];
  const int32_t* it = std::lower_bound(b, e, col);
  return (it != e && *it == col) ? K.v[it - K.ci.data()] : 0.0;
}

Strength strength(const HostCsr& K, double theta) {
  Strength S;
  S.rp.assign(K.rows + 1, 0);
  for (int64_t i = 0; i < K.rows; ++i) {
    double mx = 0.0;
    for (int64_t k = K.rp[i]; k < K.rp[i + 1]; ++k)
      if (K.ci[k] != i) mx = std::max(mx, -K.v[k]);
    const double thr = theta * mx * (1.0 + kTieRel);
    if (mx > 0.0)
      for (int64_t k = K.rp[i]; k < K.rp[i + 1]; ++k)
        if (K.ci[k] != i && -K.v[k] > thr) S.ci.push_back(K.ci[k]);
    S.rp[i + 1] = (int64_t)S.ci.size();
  }
  return S;
}

std::vector<int8_t> split(const Strength& S, int64_t n) {
  // S^T: the points that depend strongly on each point, in increasing order
  std::vector<int64_t> tp(n + 1, 0);
  for (int32_t j : S.ci) tp[j + 1]++;
  for (int64_t i = 0; i < n; ++i) tp[i + 1] += tp[i];
  std::vector<int32_t> tc(S.ci.size());
  {
    std::vector<int64_t> pos(tp.begin(), tp.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k) tc[pos[S.ci[k]]++] = (int32_t)i;
  }
  constexpr int8_t kU = -1;
  std::vector<int8_t> cf(n, kU);
  std::vector<int64_t> measure(n);
  // largest measure first, then the smallest index; stale entries skipped
  std::priority_queue<std::pair<int64_t, int64_t>> heap;
  for (int64_t i = 0; i < n; ++i) {
    measure[i] = tp[i + 1] - tp[i];
    heap.push({measure[i], -i});
  }
  std::vector<int32_t> new_f;
  int64_t left = n;
  while (left > 0 && !heap.empty()) {
    const auto top = heap.top();
    heap.pop();
    const int64_t i = -top.second;
    if (cf[i] != kU || top.first != measure[i]) continue;
    cf[i] = kC;
    --left;
    new_f.clear();
    for (int64_t k = tp[i]; k < tp[i + 1]; ++k)
      if (cf[tc[k]] == kU) new_f.push_back(tc[k]);
    for (int32_t j : new_f) {
      cf[j] = kF;
      --left;
    }
    for (int32_t j : new_f)
      for (int64_t k = S.rp[j]; k < S.rp[j + 1]; ++k) {
        const int32_t u = S.ci[k];
        if (cf[u] == kU) heap.push({++measure[u], -(int64_t)u});
      }
  }
  // second pass
  std::vector<int64_t> stamp(n, -1);  // stamp[l] == i: l in C_i
  for (int64_t i = 0; i < n; ++i) {
    if (cf[i] != kF) continue;
    for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k)
      if (cf[S.ci[k]] == kC) stamp[S.ci[k]] = i;
    int64_t tentative = -1;
    for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k) {
      const int32_t j = S.ci[k];
      if (cf[j] != kF) continue;
      bool shares = false;
      for (int64_t q = S.rp[j]; q < S.rp[j + 1] && !shares; ++q) shares = stamp[S.ci[q]] == i;
      if (shares) continue;
      if (tentative < 0) {
        tentative = j;
        stamp[j] = i;
      } else {
        cf[i] = kC;
        tentative = -1;
        break;
      }
    }
    if (tentative >= 0) cf[tentative] = kC;
  }
  return cf;
}

HostCsr interpolation(const HostCsr& K, const Strength& S, const std::vector<int8_t>& cf) {
  const int64_t n = K.rows;
  std::vector<int32_t> cidx(n, -1);
  int32_t nc = 0;
  for (int64_t i = 0; i < n; ++i)
    if (cf[i] == kC) cidx[i] = nc++;
  HostCsr P;
  P.rows = n;
  P.cols = nc;
  P.rp.assign(n + 1, 0);
  std::vector<int64_t> strong(n, -1);  // strong[m] == i: m in S_i
  std::vector<int32_t> Ci;
  struct FsTerm { int32_t m; double kim, tot; };
  std::vector<FsTerm> Fs;
  for (int64_t i = 0; i < n; ++i) {
    if (cf[i] == kC) {
      P.ci.push_back(cidx[i]);
      P.v.push_back(1.0);
      P.rp[i + 1] = (int64_t)P.ci.size();
      continue;
    }
    Ci.clear();
    for (int64_t k = S.rp[i]; k < S.rp[i + 1]; ++k) {
      strong[S.ci[k]] = i;
      if (cf[S.ci[k]] == kC) Ci.push_back(S.ci[k]);
    }
    Fs.clear();
    double den = entry(K, i, (int32_t)i);
    for (int64_t k = K.rp[i]; k < K.rp[i + 1]; ++k) {
      const int32_t m = K.ci[k];
      if (m == i) continue;
      const bool is_strong = strong[m] == i;
      if (is_strong && cf[m] == kC) continue;
      if (is_strong) {
        double tot = 0.0;
        for (int32_t l : Ci) tot += entry(K, m, l);
        if (tot != 0.0) {
          Fs.push_back({m, K.v[k], tot});
          continue;
        }
      }
      den += K.v[k];
    }
    for (int32_t j : Ci) {
      double num = entry(K, i, j);
      for (const FsTerm& t : Fs) num += t.kim * entry(K, t.m, j) / t.tot;
      P.ci.push_back(cidx[j]);
      P.v.push_back(-num / den);
    }
    P.rp[i + 1] = (int64_t)P.ci.size();
  }
  return P;
}

// threads for a host pass over `work` nonzeros (1 below a million)
static int host_threads(int64_t work) {
  if (work < (int64_t)1 << 20) return 1;
  return (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
}

// row blocks balanced by nonzeros: cut[0] = 0 <= ... <= cut[nt] = rows
static std::vector<int64_t> row_cuts(const HostCsr& A, int nt) {
  std::vector<int64_t> cut(nt + 1);
  const int64_t work = (int64_t)A.ci.size();
  for (int t = 0; t <= nt; ++t) {
    const int64_t target = work * t / nt;
    cut[t] = std::min<int64_t>(std::lower_bound(A.rp.begin(), A.rp.end(), target) - A.rp.begin(), A.rows);
  }
  cut[0] = 0;
  cut[nt] = A.rows;
  return cut;
}

// rows [r0, r1) of A B into ci / v, with the entry count of each row
static void spgemm_rows(const HostCsr& A, const HostCsr& B, int64_t r0, int64_t r1, std::vector<int32_t>& ci,
                        std::vector<double>& v, int64_t* count) {
  std::vector<double> acc(B.cols, 0.0);
  std::vector<int64_t> mark(B.cols, -1);
  std::vector<int32_t> touched;
  for (int64_t r = r0; r < r1; ++r) {
    touched.clear();
    for (int64_t a = A.rp[r]; a < A.rp[r + 1]; ++a) {
      const double va = A.v[a];
      const int32_t ka = A.ci[a];
      for (int64_t b = B.rp[ka]; b < B.rp[ka + 1]; ++b) {
        const int32_t col = B.ci[b];
        if (mark[col] != r) {
          mark[col] = r;
          acc[col] = 0.0;
          touched.push_back(col);
        }
        acc[col] += va * B.v[b];
      }
    }
    std::sort(touched.begin(), touched.end());
    int64_t k = 0;
    for (int32_t col : touched)
      if (acc[col] != 0.0) {
        ci.push_back(col);
        v.push_back(acc[col]);
        ++k;
      }
    count[r - r0] = k;
  }
}

HostCsr spgemm(const HostCsr& A, const HostCsr& B) {
  HostCsr C;
  C.rows = A.rows;
  C.cols = B.cols;
  C.rp.assign(A.rows + 1, 0);
  // contiguous row blocks on up to 16 threads (each row is computed the
  // same way whatever the split, so the result does not depend on it)
  const int nt = host_threads((int64_t)A.ci.size());
  const std::vector<int64_t> cut = row_cuts(A, nt);
  std::vector<std::vector<int32_t>> ci(nt);
  std::vector<std::vector<double>> v(nt);
  std::vector<int64_t> count(A.rows, 0);
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    if (cut[t + 1] > cut[t])
      pool.emplace_back(spgemm_rows, std::cref(A), std::cref(B), cut[t], cut[t + 1], std::ref(ci[t]), std::ref(v[t]),
                        count.data() + cut[t]);
  for (auto& th : pool) th.join();
  for (int64_t r = 0; r < A.rows; ++r) C.rp[r + 1] = C.rp[r] + count[r];
  C.ci.reserve(C.rp[A.rows]);
  C.v.reserve(C.rp[A.rows]);
  for (int t = 0; t < nt; ++t) {
    C.ci.insert(C.ci.end(), ci[t].begin(), ci[t].end());
    C.v.insert(C.v.end(), v[t].begin(), v[t].end());
  }
  return C;
}

// Stable transpose (entries of a column in increasing row order): each
// thread counts the columns of its row block, the per-thread counts give
// every (thread, column) its first slot, and each thread scatters its rows
// in order, so the result does not depend on the thread count.
HostCsr transpose(const HostCsr& A) {
  HostCsr T;
  T.rows = A.cols;
  T.cols = A.rows;
  T.rp.assign(A.cols + 1, 0);
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  // per-thread column counts: at most 2^26 entries in all
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads((int64_t)A.ci.size()),
                                                             ((int64_t)1 << 26) / std::max<int64_t>(A.cols, 1)));
  const std::vector<int64_t> cut = row_cuts(A, nt);
  std::vector<std::vector<int64_t>> cnt(nt, std::vector<int64_t>(A.cols, 0));
  auto count = [&](int t) {
    for (int64_t k = A.rp[cut[t]]; k < A.rp[cut[t + 1]]; ++k) cnt[t][A.ci[k]]++;
  };
  auto scatter = [&](int t) {
    std::vector<int64_t>& pos = cnt[t];  // first slot of (t, column)
    for (int64_t r = cut[t]; r < cut[t + 1]; ++r)
      for (int64_t k = A.rp[r]; k < A.rp[r + 1]; ++k) {
        const int64_t d = pos[A.ci[k]]++;
        T.ci[d] = (int32_t)r;
        T.v[d] = A.v[k];
      }
  };
  auto run = [&](auto&& fn) {
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(fn, t);
    fn(0);
    for (auto& th : pool) th.join();
  };
  run(count);
  int64_t off = 0;
  for (int64_t c = 0; c < A.cols; ++c) {
    T.rp[c] = off;
    for (int t = 0; t < nt; ++t) {
      const int64_t n = cnt[t][c];
      cnt[t][c] = off;
      off += n;
    }
  }
  T.rp[A.cols] = off;
  run(scatter);
  return T;
}

HostCsr galerkin(const HostCsr& K, const HostCsr& P) { return spgemm(transpose(P), spgemm(K, P)); }

HostCsr weighted_laplacian(int nv, int nh, const double* d) {
  const int64_t n = (int64_t)nv * nh, nvert = (int64_t)nh * (nv - 1);
  auto ws = [&](int i, int j) { const double v = d[i + (int64_t)j * (nv - 1)]; return v * v; };  // (i,j)-(i+1,j)
  auto we = [&](int i, int j) { const double v = d[nvert + i + (int64_t)j * nv]; return v * v; };  // (i,j)-(i,j+1)
  HostCsr K;
  K.rows = K.cols = n;
  K.rp.assign(n + 1, 0);
  for (int j = 0; j < nh; ++j)
    for (int i = 0; i < nv; ++i) {
      const int64_t p = i + (int64_t)j * nv;
      double diag = 0.0;
      if (j > 0) { K.ci.push_back((int32_t)(p - nv)); K.v.push_back(-we(i, j - 1)); diag += we(i, j - 1); }
      if (i > 0) { K.ci.push_back((int32_t)(p - 1)); K.v.push_back(-ws(i - 1, j)); diag += ws(i - 1, j); }
      const size_t at = K.ci.size();
      K.ci.push_back((int32_t)p);
      K.v.push_back(0.0);
      if (i + 1 < nv) { K.ci.push_back((int32_t)(p + 1)); K.v.push_back(-ws(i, j)); diag += ws(i, j); }
      if (j + 1 < nh) { K.ci.push_back((int32_t)(p + nv)); K.v.push_back(-we(i, j)); diag += we(i, j); }
      K.v[at] = diag;
      K.rp[p + 1] = (int64_t)K.ci.size();
    }
  return K;
}

Hierarchy hierarchy(const HostCsr& K0, int max_levels, int64_t max_coarse, double theta, bool pmis,
                    cudaStream_t s) {
  Hierarchy H;
  H.K.push_back(K0);
  while ((int)H.K.size() < max_levels && H.K.back().rows > max_coarse) {
    const HostCsr& K = H.K.back();
    const Strength S = strength(K, theta);
    const std::vector<int8_t> cf =
        pmis ? pmis_split(S, K.rows, kPmisSeed + (uint64_t)(H.K.size() - 1), s) : split(S, K.rows);
    int64_t nc = 0;
    for (int8_t f : cf) nc += f == kC;
    if (nc == 0 || nc == K.rows) break;
    H.P.push_back(interpolation(K, S, cf));
    HostCsr Kc = galerkin(K, H.P.back());
    H.K.push_back(std::move(Kc));
  }
  return H;
}

}  // namespace amg
}  // namespace lcmg
