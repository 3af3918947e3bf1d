// Launcher of the one-CTA coarse end of the V-cycle (tail.cuh).
#include "tail.cuh"
#include "tail_launch.h"

namespace lcmg {

template <class T>
void launch_vcycle_tail(const TailArgs<T>& a, cudaStream_t s) {
  klaunch(k_vcycle_tail<T>, dim3(1), dim3(tail_threads<T>()), 0, s, a);
  LCMG_LAUNCHED();
}

template void launch_vcycle_tail<float>(const TailArgs<float>&, cudaStream_t);
template void launch_vcycle_tail<double>(const TailArgs<double>&, cudaStream_t);

}  // namespace lcmg
