// Classical (Ruge-Stueben) AMG setup on the host (Sec. 3.1): strength of
// connection, the two-pass C/F split, the paper's interpolation formula and
// Galerkin products.  The paper applies it to G_L = L^T D^2 L (Sec. 3.2).
//
// The first pass is a greedy sequential algorithm by definition (each
// choice depends on every earlier one), and its result is the coarse grid,
// so it runs here on the host, once per weight vector, in O(nnz log n).
#pragma once
#include <cuda_runtime_api.h>

#include <cstdint>
#include <vector>

namespace lcmg {

struct HostCsr {
  int64_t rows = 0, cols = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;
};

namespace amg {

constexpr double kTheta = 0.25;
// a threshold tie counts as weak: -k_ij must exceed theta * max * (1 + kTieRel)
constexpr double kTieRel = 1e-10;
constexpr int8_t kC = 1, kF = 0;

// Strong connections S_i of each row (CSR pattern, increasing columns):
// j != i with -k_ij > theta * max_{m != i}(-k_im) * (1 + kTieRel).
struct Strength {
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
};

// K must have sorted column indices in each row.
Strength strength(const HostCsr& K, double theta);

// First pass: greedy selection by the measure |S_i^T| (ties: smallest
// index), each new C point's unsorted dependants become F and the unsorted
// strong connections of each new F point gain one.  Second pass, F points in
// increasing index: a strong F connection j of i without a strong connection
// into C_i is made C tentatively; a second such j makes i C instead.
std::vector<int8_t> split(const Strength& S, int64_t n);

// P (n x n_c) of the paper's formula: C points inject; F point i takes
//   w_ij = -(k_ij + sum_{m in F_i^s} k_im k_mj / sum_{l in C_i} k_ml)
//          / (k_ii + sum_{m in F_i^w} k_im)
// over its strong C connections j; coarse points numbered in fine order.
// A strong F connection whose sum over C_i is zero is lumped with F_i^w.
HostCsr interpolation(const HostCsr& K, const Strength& S, const std::vector<int8_t>& cf);

// PMIS (De Sterck, Yang and Heys 2006), the parallel replacement of the two
// passes, on the device: measure = |S_i^T| + u_i, u_i the i-th uniform
// (z >> 11) 2^-53 of the SplitMix64 stream seeded with `seed`; a point with
// no strong connection in either direction is F; then rounds in which every
// unsorted point whose (measure, index) exceeds that of each unsorted point
// it is strongly connected to (either direction) becomes C, and every
// unsorted point with a strong connection to a C point becomes F.
// Level k of a hierarchy uses seed kPmisSeed + k.
constexpr uint64_t kPmisSeed = 2306;
std::vector<int8_t> pmis_split(const Strength& S, int64_t n, uint64_t seed, cudaStream_t s);

// C = A B, rows accumulated in the order of A's and B's nonzeros, then sorted.
HostCsr spgemm(const HostCsr& A, const HostCsr& B);
HostCsr transpose(const HostCsr& A);
// P^T K P
HostCsr galerkin(const HostCsr& K, const HostCsr& P);

// L^T D^2 L of the n_v x n_h grid, d per edge (vertical edges first,
// column-major; then horizontal), rows sorted.
HostCsr weighted_laplacian(int nv, int nh, const double* d);

struct Hierarchy {
  std::vector<HostCsr> K;   // K[0] = the input, K[k+1] = P[k]^T K[k] P[k]
  std::vector<HostCsr> P;   // P[k]: level k+1 -> level k
};

// Coarsen while fewer than max_levels levels and more than max_coarse
// points remain; stop when a split keeps every point or none.  pmis: split
// by PMIS on the device (stream s) instead of the two passes.
Hierarchy hierarchy(const HostCsr& K0, int max_levels, int64_t max_coarse, double theta, bool pmis = false,
                    cudaStream_t s = nullptr);

}  // namespace amg
}  // namespace lcmg
