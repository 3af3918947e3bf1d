// Launcher of the one-cluster PCG iteration kernel (mega.cuh).
#include "mega.cuh"
#include "mega_launch.h"

namespace lcmg {

template <class T>
static int clusters_fitting(int ctas) {
  if (ctas > 8) {
    if (cudaFuncSetAttribute(k_pcg_mega<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kMegaThreads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_pcg_mega<T, false>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <class T>
int mega_cluster_ctas() {
  static int cached = -1;
  if (cached < 0) {
    cached = 0;
    for (int c : {16, 8, 4})
      if (clusters_fitting<T>(c) > 0) {
        cached = c;
        break;
      }
  }
  return cached;
}

template <class T>
void launch_pcg_mega(const MegaArgs<T>& a, int ctas, bool cache_global, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kMegaThreads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cache_global) {
    if (ctas > 8) cudaFuncSetAttribute(k_pcg_mega<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    LCMG_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_mega<T, true>, a));
  } else {
    LCMG_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_mega<T, false>, a));
  }
  LCMG_LAUNCHED();
}

template int mega_cluster_ctas<float>();
template int mega_cluster_ctas<double>();
template void launch_pcg_mega<float>(const MegaArgs<float>&, int, bool, cudaStream_t);
template void launch_pcg_mega<double>(const MegaArgs<double>&, int, bool, cudaStream_t);

}  // namespace lcmg
