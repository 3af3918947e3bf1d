// Launchers of the coarse end of the V-cycle (tail.cuh): one CTA, or one
// thread-block cluster.
#include "tail.cuh"
#include "tail_launch.h"

namespace lcmg {

template <class T>
static bool cluster_fits(int ctas) {
  if (ctas > 8 &&
      cudaFuncSetAttribute(k_vcycle_tail<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(tail_threads<T, true>());
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_vcycle_tail<T, true>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

template <class T>
int tail_cluster_ctas(int want) {
  static int cached[17] = {0};
  if (want <= 1) return 1;
  if (want > 16) want = 16;
  if (cached[want] == 0) {
    int got = 1;
    for (int c = want; c >= 2; c /= 2)
      if (cluster_fits<T>(c)) {
        got = c;
        break;
      }
    cached[want] = got;
  }
  return cached[want];
}

template <class T>
void launch_vcycle_tail(const TailArgs<T>& a, int ctas, cudaStream_t s) {
  if (ctas <= 1) {
    klaunch(k_vcycle_tail<T, false>, dim3(1), dim3(tail_threads<T>()), 0, s, a);
    LCMG_LAUNCHED();
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(tail_threads<T, true>());
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  LCMG_CUDA(cudaLaunchKernelEx(&cfg, k_vcycle_tail<T, true>, a));
  LCMG_LAUNCHED();
}

template int tail_cluster_ctas<float>(int);
template int tail_cluster_ctas<double>(int);
template void launch_vcycle_tail<float>(const TailArgs<float>&, int, cudaStream_t);
template void launch_vcycle_tail<double>(const TailArgs<double>&, int, cudaStream_t);

}  // namespace lcmg
