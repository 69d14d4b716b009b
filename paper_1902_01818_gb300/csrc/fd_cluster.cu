// a2 on the FP32 path for 2D patch interiors of small and middle size: the fast diagonalisation of
// the interior operator (Sec. 5, Eq. Ldef; L_T^{-1} = U_1 (Lambda)^{-1} U_1^T x U_0 (..) U_0^T) of one
// patch by one thread-block cluster, all four contractions in one launch.
//
// With R the patch interior of r (n1 x n0, row i1, column i0) the smoother adds
//   u_T += tau U_1 ( (U_1^T R U_0) * dinv ) U_0^T,   dinv[m][j] = 1 / (sigma + lambda_1[m] + lambda_0[j]).
// CTA c of the cluster owns the output columns J_c = [c w, c w + w) of every intermediate:
//   1) T      = R U_0[:, J_c]                   (R whole in shared memory)
//   2) X_c    = (U_1^T T) * dinv[:, J_c]        written into every CTA's copy of X (distributed
//                                               shared memory), then a cluster barrier
//   3) Y      = X U_0[J_c, :]^T                 (X whole)
//   4) u[:, J_c] += tau U_1 Y
// so the only exchange is the all-gather of X.  In a step, thread (g, i) sums output row i over the
// g-th of ks ranges of the contraction index, the groups' partial sums meeting in shared memory
// (added in group order); the row's w columns stay in registers and the contraction's B-operand
// row is read as float4 broadcasts.  The arithmetic is FP32 (as fd_small_2d<float> and the FP32
// batched steps), r read and u updated in FP64.
#include <algorithm>
#include <cstdlib>

#include <cooperative_groups.h>

#include "device.cuh"
#include "kernels.h"

namespace mgiga {
namespace dev {

namespace {

__host__ __device__ constexpr int fdc_align4(int x) { return (x + 3) & ~3; }

// the shared-memory layout of one patch (offsets in floats)
struct FdcLayout {
  int pu, pb, o_big, o_u0c, o_u0r, o_t, o_red, total;
  __host__ __device__ FdcLayout(int n0, int n1, int n1p, int wm, int ks) {
    pu = n1 | 1;  // odd row pitches: threads of a warp take consecutive rows
    pb = n0 | 1;
    o_big = fdc_align4(n1 * pu);
    o_u0c = o_big + fdc_align4(n1 * pb);
    o_u0r = o_u0c + n0 * wm;
    o_t = o_u0r + n0 * wm;
    o_red = o_t + n1 * wm;
    total = o_red + (ks - 1) * n1p * wm;
  }
};

// acc[j] += sum_{k in [kb, ke)} a(k) b[k][j], b rows of WM floats (16-byte aligned)
template <int WM, typename FA>
__device__ __forceinline__ void fdc_contract(float (&acc)[WM], FA a, const float* __restrict__ b, int kb, int ke) {
#pragma unroll 4
  for (int k = kb; k < ke; ++k) {
    const float av = a(k);
    const float4* bk = reinterpret_cast<const float4*>(b + k * WM);
#pragma unroll
    for (int v = 0; v < WM / 4; ++v) {
      const float4 bv = bk[v];
      acc[4 * v] = fmaf(av, bv.x, acc[4 * v]);
      acc[4 * v + 1] = fmaf(av, bv.y, acc[4 * v + 1]);
      acc[4 * v + 2] = fmaf(av, bv.z, acc[4 * v + 2]);
      acc[4 * v + 3] = fmaf(av, bv.w, acc[4 * v + 3]);
    }
  }
}

// the groups' partial sums of row i into group 0 (in group order); true for the threads that then
// hold the row's result.  Ends with the CTA barrier's guarantees for red.
template <int WM>
__device__ __forceinline__ bool fdc_reduce(float (&acc)[WM], float* red, int i, int g, int ks, int n1p, bool row) {
  if (g > 0 && row) {
    float4* d = reinterpret_cast<float4*>(red + ((g - 1) * n1p + i) * WM);
#pragma unroll
    for (int v = 0; v < WM / 4; ++v) d[v] = make_float4(acc[4 * v], acc[4 * v + 1], acc[4 * v + 2], acc[4 * v + 3]);
  }
  __syncthreads();
  if (g != 0 || !row) return false;
  for (int h = 1; h < ks; ++h) {
    const float4* s = reinterpret_cast<const float4*>(red + ((h - 1) * n1p + i) * WM);
#pragma unroll
    for (int v = 0; v < WM / 4; ++v) {
      const float4 x = s[v];
      acc[4 * v] += x.x;
      acc[4 * v + 1] += x.y;
      acc[4 * v + 2] += x.z;
      acc[4 * v + 3] += x.w;
    }
  }
  return true;
}

template <int WM>
__device__ __forceinline__ void fdc_zero(float (&acc)[WM]) {
#pragma unroll
  for (int j = 0; j < WM; ++j) acc[j] = 0.0f;
}

template <int WM>
__device__ __forceinline__ void fdc_store_row(const float (&acc)[WM], float* dst) {
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int v = 0; v < WM / 4; ++v) d[v] = make_float4(acc[4 * v], acc[4 * v + 1], acc[4 * v + 2], acc[4 * v + 3]);
}

template <int WM>
__global__ void __launch_bounds__(640, 1) fd_cluster_2d(const FdSmall* __restrict__ patches,
                                                         const double* __restrict__ r, double* __restrict__ u,
                                                         double tau, int ks) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) float fdc_smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const FdSmall q = patches[blockIdx.x / cs];
  const int n0 = q.n0, n1 = q.n1, N0 = q.N0;
  const int w = (n0 + cs - 1) / cs, j0 = c * w, wc = max(0, min(w, n0 - j0));
  const int n1p = blockDim.x / ks;
  const FdcLayout lo(n0, n1, n1p, WM, ks);
  float* U1s = fdc_smem;  // U_1 [n1][pu]
  float* Big = fdc_smem + lo.o_big;  // R, later X [n1][pb]
  float* U0c = fdc_smem + lo.o_u0c;  // U_0[k][j0 + jj]
  float* U0r = fdc_smem + lo.o_u0r;  // U_0[j0 + jj][k], stored [k][jj]
  float* Ts = fdc_smem + lo.o_t;     // T, X_c, Y [n1][WM]
  float* red = fdc_smem + lo.o_red;  // partial sums [ks - 1][n1p][WM]
  const float* gU0 = static_cast<const float*>(q.U0);
  const float* gU1 = static_cast<const float*>(q.U1);
  const float* gD = static_cast<const float*>(q.dinv);
  const double* rg = r + q.ibase;
  const int tid = threadIdx.x, nthr = blockDim.x;
  // operands into shared memory, eight independent loads in flight per thread
  constexpr int LU = 8;
  for (int x0 = tid; x0 < n1 * n1; x0 += LU * nthr) {
    float v[LU];
#pragma unroll
    for (int j = 0; j < LU; ++j) v[j] = x0 + j * nthr < n1 * n1 ? __ldg(gU1 + x0 + j * nthr) : 0.0f;
#pragma unroll
    for (int j = 0; j < LU; ++j) {
      const int x = x0 + j * nthr;
      if (x < n1 * n1) U1s[(x / n1) * lo.pu + x % n1] = v[j];
    }
  }
  for (int x0 = tid; x0 < n1 * n0; x0 += LU * nthr) {
    double v[LU];
#pragma unroll
    for (int j = 0; j < LU; ++j) {
      const int x = x0 + j * nthr;
      v[j] = x < n1 * n0 ? __ldg(rg + (int64_t)(x / n0) * N0 + x % n0) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < LU; ++j) {
      const int x = x0 + j * nthr;
      if (x < n1 * n0) Big[(x / n0) * lo.pb + x % n0] = (float)v[j];
    }
  }
  for (int x0 = tid; x0 < n0 * WM; x0 += (LU / 2) * nthr) {
    float vc[LU / 2], vr[LU / 2];
#pragma unroll
    for (int j = 0; j < LU / 2; ++j) {
      const int x = x0 + j * nthr, k = x / WM, jj = x % WM;
      const bool ok = x < n0 * WM && jj < wc;
      vc[j] = ok ? __ldg(gU0 + k * n0 + j0 + jj) : 0.0f;
      vr[j] = ok ? __ldg(gU0 + (j0 + jj) * n0 + k) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < LU / 2; ++j) {
      const int x = x0 + j * nthr;
      if (x < n0 * WM) {
        U0c[x] = vc[j];
        U0r[x] = vr[j];
      }
    }
  }
  __syncthreads();
  const int i = tid % n1p, g = tid / n1p;
  const bool row = i < n1;
  const int kb0 = g * n0 / ks, ke0 = (g + 1) * n0 / ks;  // contraction ranges over n0 (steps 1, 3)
  const int kb1 = g * n1 / ks, ke1 = (g + 1) * n1 / ks;  // and over n1 (steps 2, 4)
  float acc[WM];
  // 1) T = R U_0[:, J_c]
  fdc_zero(acc);
  if (row) fdc_contract(acc, [&](int k) { return Big[i * lo.pb + k]; }, U0c, kb0, ke0);
  if (fdc_reduce(acc, red, i, g, ks, n1p, row)) fdc_store_row(acc, Ts + i * WM);
  __syncthreads();
  // this CTA has read R for the last time: the others may overwrite its Big with X
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  // 2) X_c = (U_1^T T) * dinv[:, J_c]
  fdc_zero(acc);
  if (row) fdc_contract(acc, [&](int k) { return U1s[k * lo.pu + i]; }, Ts, kb1, ke1);
  if (fdc_reduce(acc, red, i, g, ks, n1p, row)) {
#pragma unroll
    for (int jj = 0; jj < WM; ++jj) acc[jj] = jj < wc ? acc[jj] * gD[i * n0 + j0 + jj] : 0.0f;
    fdc_store_row(acc, Ts + i * WM);  // every thread has left step 2's loop (barrier in fdc_reduce)
  }
  __syncthreads();
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  // X_c into every CTA's X (its own included), then the cluster barrier publishes the stores
  for (int rr = 0; rr < cs; ++rr) {
    float* dst = cluster.map_shared_rank(Big, rr);
    for (int x = tid; x < n1 * wc; x += nthr) {
      const int m = x / wc, jj = x - m * wc;
      dst[m * lo.pb + j0 + jj] = Ts[m * WM + jj];
    }
  }
  cluster.sync();
  // 3) Y = X U_0[J_c, :]^T
  fdc_zero(acc);
  if (row) fdc_contract(acc, [&](int k) { return Big[i * lo.pb + k]; }, U0r, kb0, ke0);
  if (fdc_reduce(acc, red, i, g, ks, n1p, row)) fdc_store_row(acc, Ts + i * WM);
  __syncthreads();
  // 4) u[:, J_c] += tau U_1 Y
  fdc_zero(acc);
  if (row) fdc_contract(acc, [&](int k) { return U1s[i * lo.pu + k]; }, Ts, kb1, ke1);
  if (fdc_reduce(acc, red, i, g, ks, n1p, row)) {
    double* ug = u + q.ibase + (int64_t)i * N0 + j0;
#pragma unroll
    for (int jj = 0; jj < WM; ++jj)
      if (jj < wc) ug[jj] += tau * (double)acc[jj];
  }
}

constexpr int kFdcSmemMax = 227 * 1024;

void* fdc_kernel(int wm) {
  switch (wm) {
    case 4: return (void*)fd_cluster_2d<4>;
    case 8: return (void*)fd_cluster_2d<8>;
    case 12: return (void*)fd_cluster_2d<12>;
    case 16: return (void*)fd_cluster_2d<16>;
    case 20: return (void*)fd_cluster_2d<20>;
    default: return nullptr;
  }
}

// clusters of this shape that can be resident at once (0: none, or the query failed)
int fdc_resident(const FdClusterShape& s) {
  void* fn = fdc_kernel(s.wm);
  if (!fn) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kFdcSmemMax) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(s.cs);
  cfg.blockDim = dim3(s.threads);
  cfg.dynamicSmemBytes = s.smem;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = s.cs;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

bool fd_cluster_shape(int n0max, int n1max, int npatch, FdClusterShape* out) {
  if (n0max <= 0 || n1max <= 0 || n1max > 640) return false;
  const int n1p = (n1max + 31) / 32 * 32;
  FdClusterShape best{};
  bool found = false;
  // the largest cluster whose clusters for all patches are resident at once (else the one with
  // the most resident clusters): more CTAs per patch, fewer columns each
  int only = 0;  // MGIGA_FD_CLUSTER_CS: one cluster size (2, 4, 8, 16) for tuning and tests
  if (const char* env = std::getenv("MGIGA_FD_CLUSTER_CS")) only = std::atoi(env);
  for (int cs : {16, 8, 4, 2}) {
    if (only > 0 && cs != only) continue;
    const int w = (n0max + cs - 1) / cs;
    const int wm = (w + 3) / 4 * 4;
    if (wm > 20) break;  // fewer CTAs only widens the slices further
    for (int ks = std::min(4, 640 / n1p); ks >= 1; --ks) {  // at most 640 threads (the launch bound)
      const FdcLayout lo(n0max, n1max, n1p, wm, ks);
      const int smem = lo.total * (int)sizeof(float);
      if (smem > kFdcSmemMax) continue;
      FdClusterShape s{cs, wm, ks, n1p * ks, smem, 0};
      s.resident = fdc_resident(s);
      if (s.resident <= 0) break;
      if (!found || std::min(s.resident, npatch) > std::min(best.resident, npatch)) {
        best = s;
        found = true;
      }
      break;
    }
    if (found && best.resident >= npatch) break;
  }
  if (found) *out = best;
  return found;
}

cudaError_t launch_fd_cluster(int npatch, const FdClusterShape& s, cudaStream_t st, const FdSmall* patches,
                              const double* r, double* u, double tau) {
  if (npatch == 0) return cudaSuccess;
  void* fn = fdc_kernel(s.wm);
  if (!fn) return cudaErrorInvalidValue;
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(npatch * s.cs);
  cfg.blockDim = dim3(s.threads);
  cfg.dynamicSmemBytes = s.smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = s.cs;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int ks = s.ks;
  void* args[] = {(void*)&patches, (void*)&r, (void*)&u, (void*)&tau, (void*)&ks};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace dev
}  // namespace mgiga
