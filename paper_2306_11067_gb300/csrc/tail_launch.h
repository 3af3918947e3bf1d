// Declaration of the one-CTA coarse V-cycle launcher (tail.cu).
#pragma once
#include "common.cuh"

namespace lcmg {

template <class T>
struct TailArgs;

template <class T>
void launch_vcycle_tail(const TailArgs<T>& a, cudaStream_t s);

}  // namespace lcmg
