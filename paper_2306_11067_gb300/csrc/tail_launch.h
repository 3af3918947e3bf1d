// Declarations of the coarse V-cycle launchers (tail.cu).
#pragma once
#include "common.cuh"

namespace lcmg {

template <class T>
struct TailArgs;

// cluster size the tail runs with: the largest of want, want/2, ... >= 2
// whose cluster fits on the device, else 1 (one CTA)
template <class T>
int tail_cluster_ctas(int want);

// ctas = 1: one CTA; ctas > 1: one cluster of that many CTAs
template <class T>
void launch_vcycle_tail(const TailArgs<T>& a, int ctas, cudaStream_t s);

}  // namespace lcmg
