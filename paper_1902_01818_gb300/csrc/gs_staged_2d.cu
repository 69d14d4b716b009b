// Instances of the patch-parallel Gauss-Seidel phase for 2D patches, and the host side (cluster fit
// query, launch) of both dimensions.
#include "gs_staged.cuh"

namespace mgiga {
namespace dev {

void* gs_staged_ptr_2d(int p, int tpr) { return gs_staged_ptr_dim<2>(p, tpr); }

namespace {
constexpr int kStagedSmemMax = 225 * 1024;

static void* gs_staged_ptr(int d, int p, int tpr) {
  return d == 2 ? gs_staged_ptr_2d(p, tpr) : gs_staged_ptr_3d(p, tpr);
}


}  // namespace

bool gs_staged_fits(int d, int p, int tpr, int csize, int smem, int threads) {
  void* fn = gs_staged_ptr(d, p, tpr);
  if (!fn) return false;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
  // the attribute belongs to the kernel, not to a launch: always allow the
  // largest amount any level may ask for (kStagedSmemMax)
  if (smem > kStagedSmemMax ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = csize;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters > 0;
}

cudaError_t launch_gs_staged(int d, int p, int nclusters, int smem, cudaStream_t st, const GsStagedArgs& a) {
  if (nclusters <= 0) return cudaSuccess;
  void* fn = gs_staged_ptr(d, p, a.tpr);
  if (!fn) return cudaErrorInvalidValue;
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * a.csize);
  cfg.blockDim = dim3(a.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = a.csize;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  GsStagedArgs arg = a;
  void* args[] = {&arg};
  return cudaLaunchKernelExC(&cfg, fn, args);
}


}  // namespace dev
}  // namespace mgiga
