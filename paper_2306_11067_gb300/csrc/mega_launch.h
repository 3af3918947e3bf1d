// Declarations of the one-cluster PCG iteration launcher (mega.cu).
#pragma once
#include "common.cuh"

namespace lcmg {

constexpr int kMegaMaxLevels = 16;
constexpr int kMegaMaxCtas = 16;

template <class T>
struct MegaArgs;

// CTAs per cluster this GPU accepts for the kernel (16, 8 or 4), 0 if none
template <class T>
int mega_cluster_ctas();

template <class T>
void launch_pcg_mega(const MegaArgs<T>& a, int ctas, bool cache_global, cudaStream_t s);

}  // namespace lcmg
