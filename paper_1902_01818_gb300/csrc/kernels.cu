// CUDA kernels of the V-cycle and of PCG (FP64 path), for sm_103a.
//
//   band_apply      residual r = f - A u / product A u on the patch band (a1)
//   cross_apply     SIPG cross-patch couplings (a1')
//   shared_reduce   sums / copies of DoFs shared by conforming patches (a1')
//   restrict_band   f_c = P^T (w r) per patch, tensor-product children (a5)
//   prolong_band    u_f += P e_c per patch, tensor-product parents (a6)
//   gemm_tiled      batched strided GEMM of the fast-diagonalisation
//                   contractions, with the eigenvalue-sum division and the
//                   damped update fused into the epilogue (a2)
//   piece_apply     interface-piece and coarse solves, z = Z r (a3, a7)
//   gs_sweep_coop   a whole multicolour Gauss-Seidel sweep, one cooperative launch (a4)
//   dot / cg_*      deterministic reductions and vector updates of PCG (a8)
#include <cstdio>
#include <type_traits>

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"
#include "ptx.cuh"

namespace mgiga {
namespace dev {

// ---------------------------------------------------------------------------
// a1: band residual / product
// ---------------------------------------------------------------------------
// One thread per row.  The band coefficients of offset o for consecutive rows
// are consecutive (coalesced); the u neighbours are read through L1/L2.
// MODE 0: out = f - A u;  MODE 1: out = A u.
template <int D, int P, int MODE>
__global__ void __launch_bounds__(kTile) band_apply(const Tile* __restrict__ tiles,
                                                    const PatchMeta* __restrict__ patches,
                                                    const double* __restrict__ band, int64_t nloc,
                                                    const double* __restrict__ u,
                                                    const double* __restrict__ f,
                                                    double* __restrict__ out) {
  const Tile t = tiles[blockIdx.x];
  if ((int)threadIdx.x >= t.count) return;
  const int64_t pos = t.start + threadIdx.x;
  const PatchMeta pm = patches[t.patch];
  const int64_t s1 = pm.N[0], s2 = (int64_t)pm.N[0] * pm.N[1];
  constexpr int W = 2 * P + 1;
  double acc = 0.0;
  const double* b = band + pos;
  const double* uc = u + pos;
#pragma unroll 1
  for (int o2 = 0; o2 < (D == 3 ? W : 1); ++o2) {
    const int64_t off2 = D == 3 ? (int64_t)(o2 - P) * s2 : 0;
#pragma unroll 1
    for (int o1 = 0; o1 < W; ++o1) {
      const double* ur = uc + off2 + (int64_t)(o1 - P) * s1 - P;
      const double* br = b + (int64_t)((o2 * W + o1) * W) * nloc;
#pragma unroll
      for (int o0 = 0; o0 < W; ++o0) acc = fma(__ldg(br + (int64_t)o0 * nloc), ur[o0], acc);
    }
  }
  if (MODE == 0) out[pos] = f[pos] - acc;
  else out[pos] = acc;
}

// a1 in FP32, for the residuals inside the mixed-precision cycle (they feed
// the FP32 smoothers and the restriction): out = f - A u with FP32
// coefficients band32[o * nloc + pos] and FP32 arithmetic, out in FP64.  A
// row group is kRowsF32 consecutive rows of a tile; for every (o2, o1) line a
// thread reads the W + kRowsF32 - 1 consecutive u values the group needs,
// converts each once, and applies the W coefficients of each row.  G threads
// share a group (lines j, j + G, ..; thread index = j 64 + group, so a warp
// reads 32 consecutive groups), their sums added in a fixed order through
// shared memory.  band32 carries kRowsF32 padding floats at its end; u has
// zero guards.
constexpr int kRowsF32 = 4;
template <int D, int P, int G>
__global__ void __launch_bounds__(kTile / kRowsF32 * G) band_residual_f32(const Tile* __restrict__ tiles,
                                                                      const PatchMeta* __restrict__ patches,
                                                                      const float* __restrict__ band32,
                                                                      int64_t nloc, const double* __restrict__ u,
                                                                      const double* __restrict__ f,
                                                                      double* __restrict__ out) {
  constexpr int NG = kTile / kRowsF32;  // row groups per tile
  __shared__ float red[G > 1 ? G - 1 : 1][NG][kRowsF32];
  const Tile t = tiles[blockIdx.x];
  const int rg = threadIdx.x % NG, j = threadIdx.x / NG;
  const int r0 = rg * kRowsF32;
  const bool live = r0 < t.count;
  const int64_t pos0 = t.start + (live ? r0 : 0);
  const PatchMeta pm = patches[t.patch];
  const int64_t s1 = pm.N[0], s2 = (int64_t)pm.N[0] * pm.N[1];
  constexpr int W = 2 * P + 1;
  constexpr int U = W + kRowsF32 - 1;
  constexpr int NL = D == 3 ? W * W : W;  // (o2, o1) lines
  float acc[kRowsF32];
#pragma unroll
  for (int q = 0; q < kRowsF32; ++q) acc[q] = 0.0f;
  if (live) {
    const float* b = band32 + pos0;
    const double* uc = u + pos0;
#pragma unroll 1
    for (int line = j; line < NL; line += G) {
      const int o1 = line % W, o2 = line / W;
      const double* ur = uc + (D == 3 ? (int64_t)(o2 - P) * s2 : 0) + (int64_t)(o1 - P) * s1 - P;
      float uf[U];
#pragma unroll
      for (int i = 0; i < U; ++i) uf[i] = (float)__ldg(ur + i);
      const float* br = b + (int64_t)(line * W) * nloc;
#pragma unroll
      for (int o0 = 0; o0 < W; ++o0)
#pragma unroll
        for (int q = 0; q < kRowsF32; ++q) acc[q] = fmaf(__ldg(br + (int64_t)o0 * nloc + q), uf[q + o0], acc[q]);
    }
  }
  if (G > 1) {
    if (j > 0)
#pragma unroll
      for (int q = 0; q < kRowsF32; ++q) red[j - 1][rg][q] = acc[q];
    __syncthreads();
    if (j > 0) return;
#pragma unroll
    for (int jj = 0; jj < G - 1; ++jj)
#pragma unroll
      for (int q = 0; q < kRowsF32; ++q) acc[q] += red[jj][rg][q];
  }
  if (!live) return;
  const int nq = min(kRowsF32, t.count - r0);
  for (int q = 0; q < nq; ++q) out[pos0 + q] = f[pos0 + q] - (double)acc[q];
}

// a1': out[row] -= (MODE 0) or += (MODE 1) sum_j C[row, j] u[j]; a warp per row
template <int MODE>
__global__ void cross_apply(int nx, const int64_t* __restrict__ x_row, const int* __restrict__ x_ptr,
                            const int64_t* __restrict__ x_col, const double* __restrict__ x_val,
                            const double* __restrict__ u, double* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nx) return;
  double s = 0.0;
  for (int j = x_ptr[w] + lane; j < x_ptr[w + 1]; j += 32) s = fma(x_val[j], u[x_col[j]], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    if (MODE == 0) out[x_row[w]] -= s;
    else out[x_row[w]] += s;
  }
}

// conforming shared DoFs.  mode 0 (residual): total = sum_c v[c] - (m-1) f[c0];
// mode 1 (sum of partial products); mode 2 (copy the owner value)
__global__ void shared_reduce(int nsh, const int* __restrict__ sh_ptr, const int64_t* __restrict__ sh_pos,
                              double* __restrict__ v, const double* __restrict__ f, int mode) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nsh) return;
  const int b = sh_ptr[c], e = sh_ptr[c + 1];
  double total;
  if (mode == 2) {
    total = v[sh_pos[b]];
  } else {
    total = 0.0;
    for (int i = b; i < e; ++i) total += v[sh_pos[i]];
    if (mode == 0) total -= (double)(e - b - 1) * f[sh_pos[b]];
  }
  for (int i = b; i < e; ++i) v[sh_pos[i]] = total;
}

// ---------------------------------------------------------------------------
// a5 / a6: transfers, tensor products of the 1D knot-insertion matrices
// ---------------------------------------------------------------------------
// f_c[I] = sum_{i} prod_a P_a[i_a, I_a] (w r)[i], children i_a of I_a from the
// tables; coarse Dirichlet entries are left 0.  T: arithmetic type (double;
// float inside the mixed-precision cycle, where the transfers only feed the
// preconditioner -- FP64 runs at 1/64 of the FP32 rate on this part).
template <int D, typename T>
__global__ void __launch_bounds__(kTile) restrict_band(
    const Tile* __restrict__ tiles, const PatchMeta* __restrict__ pc, const PatchMeta* __restrict__ pf,
    const XferMeta* __restrict__ xm, const int* __restrict__ ch_start, const double* __restrict__ ch_val,
    int cw, const double* __restrict__ r, const double* __restrict__ w, const int* __restrict__ c_l2g,
    double* __restrict__ out) {
  const Tile t = tiles[blockIdx.x];
  if ((int)threadIdx.x >= t.count) return;
  const int64_t pos = t.start + threadIdx.x;
  const int k = t.patch;
  if (c_l2g[pos] < 0) { out[pos] = 0.0; return; }
  const PatchMeta mc = pc[k], mf = pf[k];
  int64_t rem = pos - mc.off;
  int I[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) { I[a] = (int)(rem % mc.N[a]); rem /= mc.N[a]; }
  int st[3] = {0, 0, 0};
  const double* cv[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < D; ++a) {
    const XferMeta x = xm[k * 3 + a];
    st[a] = ch_start[x.ch_off + I[a]];
    cv[a] = ch_val + (x.ch_off + I[a]) * cw;
  }
  T s = 0;
  for (int t2 = 0; t2 < (D == 3 ? cw : 1); ++t2) {
    const T c2 = D == 3 ? (T)cv[2][t2] : (T)1;
    if (c2 == (T)0) continue;
    const int i2 = D == 3 ? st[2] + t2 : 0;
    for (int t1 = 0; t1 < cw; ++t1) {
      const T c1 = (T)cv[1][t1] * c2;
      if (c1 == (T)0) continue;
      const int i1 = st[1] + t1;
      const int64_t rowb = mf.off + (int64_t)mf.N[0] * (i1 + (int64_t)mf.N[1] * i2);
      T s1 = 0;
      for (int t0 = 0; t0 < cw; ++t0) {
        const T c0 = (T)cv[0][t0];
        if (c0 == (T)0) continue;
        const int64_t fp = rowb + st[0] + t0;
        const T v = (T)(w ? w[fp] * r[fp] : r[fp]);
        s1 = fma(c0, v, s1);
      }
      s = fma(c1, s1, s);
    }
  }
  out[pos] = (double)s;
}

// u_f[i] += sum_I prod_a P_a[i_a, I_a] e_c[I]  (T: arithmetic type, as for the restriction)
template <int D, typename T>
__global__ void __launch_bounds__(kTile) prolong_band(
    const Tile* __restrict__ tiles, const PatchMeta* __restrict__ pf, const PatchMeta* __restrict__ pc,
    const XferMeta* __restrict__ xm, const int* __restrict__ par_start, const double* __restrict__ par_val,
    int pw, const double* __restrict__ e, double* __restrict__ u) {
  const Tile t = tiles[blockIdx.x];
  if ((int)threadIdx.x >= t.count) return;
  const int64_t pos = t.start + threadIdx.x;
  const int k = t.patch;
  const PatchMeta mf = pf[k], mc = pc[k];
  int64_t rem = pos - mf.off;
  int i[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) { i[a] = (int)(rem % mf.N[a]); rem /= mf.N[a]; }
  int st[3] = {0, 0, 0};
  const double* pv[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < D; ++a) {
    const XferMeta x = xm[k * 3 + a];
    st[a] = par_start[x.par_off + i[a]];
    pv[a] = par_val + (x.par_off + i[a]) * pw;
  }
  T s = 0;
  for (int t2 = 0; t2 < (D == 3 ? pw : 1); ++t2) {
    const T c2 = D == 3 ? (T)pv[2][t2] : (T)1;
    if (c2 == (T)0) continue;
    const int I2 = D == 3 ? st[2] + t2 : 0;
    for (int t1 = 0; t1 < pw; ++t1) {
      const T c1 = (T)pv[1][t1] * c2;
      if (c1 == (T)0) continue;
      const int I1 = st[1] + t1;
      const int64_t rowb = mc.off + (int64_t)mc.N[0] * (I1 + (int64_t)mc.N[1] * I2);
      T s1 = 0;
      for (int t0 = 0; t0 < pw; ++t0) {
        const T c0 = (T)pv[0][t0];
        if (c0 == (T)0) continue;
        s1 = fma(c0, (T)e[rowb + st[0] + t0], s1);
      }
      s = fma(c1, s1, s);
    }
  }
  u[pos] += (double)s;
}

// Mode-wise transfers of 2D patches (the 1D knot-insertion matrices applied one
// direction at a time, Sec. 4): a CTA owns a block of rows along xi_1 of the
// output.  Restriction: the fine rows the block's children span are first
// contracted along xi_0 into shared memory, t[i_1][I_0] = sum_{i_0} P_0[i_0, I_0]
// (w r)[i_1][i_0], then along xi_1, f_c[I_1][I_0] = sum_{i_1} P_1[i_1, I_1] t[i_1][I_0];
// prolongation the same with the parents.  ~2 (p + 2) products per output instead
// of (p + 2)^2, the same summation order as restrict_band / prolong_band (so the
// FP64 results are identical).  blocks: (patch, first row, end row, -).
template <typename T>
__global__ void __launch_bounds__(256) restrict_mw2(const int4* __restrict__ blocks, const PatchMeta* __restrict__ pc,
                                                    const PatchMeta* __restrict__ pf, const XferMeta* __restrict__ xm,
                                                    const int* __restrict__ ch_start, const double* __restrict__ ch_val,
                                                    int cw, const double* __restrict__ r, const double* __restrict__ w,
                                                    const int* __restrict__ c_l2g, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char xsm[];
  T* t = reinterpret_cast<T*>(xsm);
  const int4 b = blocks[blockIdx.x];
  const int k = b.x, I1a = b.y, I1b = b.z;
  const PatchMeta mc = pc[k], mf = pf[k];
  const XferMeta x0 = xm[k * 3], x1 = xm[k * 3 + 1];
  const int N0f = mf.N[0], N1f = mf.N[1], N0c = mc.N[0];
  const int lo = ch_start[x1.ch_off + I1a];
  const int hi = min(N1f, ch_start[x1.ch_off + I1b - 1] + cw);
  for (int e = threadIdx.x; e < (hi - lo) * N0c; e += blockDim.x) {
    const int ii = e / N0c, I0 = e - ii * N0c;
    const int s0 = ch_start[x0.ch_off + I0];
    const double* cv = ch_val + (x0.ch_off + I0) * (int64_t)cw;
    const int64_t rowb = mf.off + (int64_t)N0f * (lo + ii);
    T acc = 0;
    for (int t0 = 0; t0 < cw && s0 + t0 < N0f; ++t0) {
      const int64_t fp = rowb + s0 + t0;
      acc = fma((T)cv[t0], (T)(w ? w[fp] * r[fp] : r[fp]), acc);
    }
    t[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (I1b - I1a) * N0c; e += blockDim.x) {
    const int dI = e / N0c, I0 = e - dI * N0c, I1 = I1a + dI;
    const int64_t pos = mc.off + (int64_t)I1 * N0c + I0;
    if (c_l2g[pos] < 0) { out[pos] = 0.0; continue; }
    const int s1 = ch_start[x1.ch_off + I1];
    const double* cv = ch_val + (x1.ch_off + I1) * (int64_t)cw;
    T acc = 0;
    for (int t1 = 0; t1 < cw && s1 + t1 < hi; ++t1) acc = fma((T)cv[t1], t[(s1 + t1 - lo) * N0c + I0], acc);
    out[pos] = (double)acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) prolong_mw2(const int4* __restrict__ blocks, const PatchMeta* __restrict__ pf,
                                                   const PatchMeta* __restrict__ pc, const XferMeta* __restrict__ xm,
                                                   const int* __restrict__ par_start, const double* __restrict__ par_val,
                                                   int pw, const double* __restrict__ e, double* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char xsm[];
  T* s = reinterpret_cast<T*>(xsm);
  const int4 b = blocks[blockIdx.x];
  const int k = b.x, i1a = b.y, i1b = b.z;
  const PatchMeta mf = pf[k], mc = pc[k];
  const XferMeta x0 = xm[k * 3], x1 = xm[k * 3 + 1];
  const int N0f = mf.N[0], N0c = mc.N[0], N1c = mc.N[1];
  const int lo = par_start[x1.par_off + i1a];
  const int hi = min(N1c, par_start[x1.par_off + i1b - 1] + pw);
  for (int q = threadIdx.x; q < (hi - lo) * N0f; q += blockDim.x) {
    const int ii = q / N0f, i0 = q - ii * N0f;
    const int s0 = par_start[x0.par_off + i0];
    const double* pv = par_val + (x0.par_off + i0) * (int64_t)pw;
    const int64_t rowb = mc.off + (int64_t)N0c * (lo + ii);
    T acc = 0;
    for (int t0 = 0; t0 < pw && s0 + t0 < N0c; ++t0) acc = fma((T)pv[t0], (T)e[rowb + s0 + t0], acc);
    s[q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < (i1b - i1a) * N0f; q += blockDim.x) {
    const int di = q / N0f, i0 = q - di * N0f, i1 = i1a + di;
    const int s1 = par_start[x1.par_off + i1];
    const double* pv = par_val + (x1.par_off + i1) * (int64_t)pw;
    T acc = 0;
    for (int t1 = 0; t1 < pw && s1 + t1 < hi; ++t1) acc = fma((T)pv[t1], s[(s1 + t1 - lo) * N0f + i0], acc);
    u[mf.off + (int64_t)i1 * N0f + i0] += (double)acc;
  }
}

// ---------------------------------------------------------------------------
// a2: batched FP64 GEMM for the fast-diagonalisation contractions
// ---------------------------------------------------------------------------
constexpr int GBK = 16;

__device__ __forceinline__ int64_t gcol(const GemmTask& g, int n) {
  return (int64_t)(n / g.ndiv) * g.nhi + (n % g.ndiv);
}

template <typename T>
__device__ __forceinline__ T ldt(const void* p, int64_t i, int t) {
  return t ? (T) static_cast<const float*>(p)[i] : (T) static_cast<const double*>(p)[i];
}

// BM x BM output tile per CTA of 256 threads (16 x 16), each thread a
// (BM/16) x (BM/16) micro-tile of rows ty T.. and columns tx T.. (T = BM/16);
// Acc is the arithmetic type (double: the FP64 path, float: the FP32 path of
// the mixed-precision cycle), TA / TB the element types of A / B in memory
// (the first step of the FP32 path reads the FP64 residual).  K is consumed
// in slabs of GBK, staged into shared memory by element-wise asynchronous
// copies (zero-filled outside the matrix) through a ring of kGemmStages
// slabs, so that the global-memory latency of slab k + 2 overlaps the FMAs of
// slab k.  In FP64 the FMA pipe (2 DFMA/clk/SM on this part) is the bound, so
// BM = 32 (more tiles in flight, less work on ragged edges); FP32 uses BM = 64
// for reuse.
// Stages: FP64 3 (the FMA pipe is the bound), FP32 6 (~1 us of global latency
// covered by 5 slabs in flight).
constexpr int kGemmStagesF64 = 3, kGemmStagesF32 = 6;

template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
               "r"(valid ? BYTES : 0)
               : "memory");
}

template <int BM, typename Acc, typename TA, typename TB, int STAGES>
struct GemmSmem {
  static constexpr int PA = BM + 16 / (int)sizeof(TA);  // row pitches: 16-byte multiples
  static constexpr int PB = BM + 16 / (int)sizeof(TB);
  static constexpr int PC = BM + 16 / (int)sizeof(Acc);
  static constexpr bool CVT = !std::is_same<TA, Acc>::value;  // A converted once per slab into Ac
  static constexpr size_t a_bytes = (size_t)STAGES * GBK * PA * sizeof(TA);
  static constexpr size_t b_bytes = (size_t)STAGES * GBK * PB * sizeof(TB);
  static constexpr size_t c_bytes = CVT ? (size_t)2 * GBK * PC * sizeof(Acc) : 0;
  static constexpr size_t bytes = a_bytes + b_bytes + c_bytes;
};

template <int BM, typename Acc, typename TA, typename TB, int STAGES>
__global__ void __launch_bounds__(256) gemm_tiled(const GemmTask* __restrict__ tasks,
                                                  const GemmItem* __restrict__ items) {
  constexpr int kGemmStages = STAGES;
  using SM = GemmSmem<BM, Acc, TA, TB, STAGES>;
  constexpr int T = BM / 16;
  constexpr int PA = SM::PA, PB = SM::PB, PC = SM::PC;
  constexpr bool CVT = SM::CVT;
  extern __shared__ __align__(16) unsigned char gemm_smem[];
  auto As = reinterpret_cast<TA(*)[GBK][PA]>(gemm_smem);
  auto Bs = reinterpret_cast<TB(*)[GBK][PB]>(gemm_smem + SM::a_bytes);
  auto Ac = reinterpret_cast<Acc(*)[GBK][PC]>(gemm_smem + SM::a_bytes + SM::b_bytes);
  const GemmItem it = items[blockIdx.x];
  const GemmTask g = tasks[it.task];
  const TA* Ag = static_cast<const TA*>(g.A) + it.z * g.sA;
  const TB* Bg = static_cast<const TB*>(g.B) + it.z * g.sB;
  const int64_t oC = it.z * g.sC;
  const int m0 = it.tm * BM, n0 = it.tn * BM;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nk = (g.K + GBK - 1) / GBK;
  // this thread's elements of a slab: A element l at (mA + l dmA, kA + l dkA), B element l at (nB + l dnB, kB + l dkB)
  int mA, kA, dmA, dkA, nB, kB, dnB, dkB;
  if (g.transA) { mA = tid % BM; kA = tid / BM; dmA = 0; dkA = 256 / BM; }
  else { kA = tid & 15; mA = tid >> 4; dmA = 16; dkA = 0; }
  if (g.transB) { kB = tid & 15; nB = tid >> 4; dnB = 16; dkB = 0; }
  else { nB = tid % BM; kB = tid / BM; dnB = 0; dkB = 256 / BM; }
  const int64_t sAm = g.transA ? 1 : g.lda, sAk = g.transA ? g.lda : 1;
  const int64_t sBn = g.transB ? g.ldb : 1, sBk = g.transB ? 1 : g.ldb;
  auto load = [&](int s, int kt) {
    const int k0 = kt * GBK;
#pragma unroll
    for (int l = 0; l < T; ++l) {
      {
        const int mm = mA + l * dmA, kk = kA + l * dkA;
        const int m = m0 + mm, k = k0 + kk;
        const bool ok = m < g.M && k < g.K;
        cp_async_elem<sizeof(TA)>(&As[s][kk][mm], ok ? Ag + m * sAm + k * sAk : Ag, ok);
      }
      {
        const int nn = nB + l * dnB, kk = kB + l * dkB;
        const int n = n0 + nn, k = k0 + kk;
        const bool ok = n < g.N && k < g.K;
        cp_async_elem<sizeof(TB)>(&Bs[s][kk][nn], ok ? Bg + n * sBn + k * sBk : Bg, ok);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
#pragma unroll
  for (int s = 0; s < kGemmStages - 1; ++s) {
    if (s < nk) load(s, s);
    else asm volatile("cp.async.commit_group;" ::: "memory");
  }
  Acc acc[T][T];
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int j = 0; j < T; ++j) acc[i][j] = 0;
  for (int kt = 0; kt < nk; ++kt) {
    asm volatile("cp.async.wait_group %0;" ::"n"(kGemmStages - 2) : "memory");
    const int s = kt % kGemmStages;
    if constexpr (CVT) {  // this thread's own elements of slab kt have landed: convert them once
#pragma unroll
      for (int l = 0; l < T; ++l) {
        const int mm = mA + l * dmA, kk = kA + l * dkA;
        Ac[kt & 1][kk][mm] = (Acc)As[s][kk][mm];
      }
    }
    __syncthreads();  // slab kt visible to all; slab kt - 1 no longer read
    const int nxt = kt + kGemmStages - 1;
    if (nxt < nk) load(nxt % kGemmStages, nxt);
    else asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      Acc a[T], b[T];
#pragma unroll
      for (int i = 0; i < T; ++i) a[i] = CVT ? (Acc)Ac[kt & 1][kk][ty * T + i] : (Acc)As[s][kk][ty * T + i];
#pragma unroll
      for (int j = 0; j < T; ++j) b[j] = (Acc)Bs[s][kk][tx * T + j];
#pragma unroll
      for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
  for (int i = 0; i < T; ++i) {
    const int m = m0 + ty * T + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < T; ++j) {
      const int n = n0 + tx * T + j;
      if (n >= g.N) continue;
      const int64_t ci = oC + (int64_t)m * g.ldc + gcol(g, n);
      Acc v = acc[i][j];
      if (g.epi == 1) v *= static_cast<const Acc*>(g.dinv)[(int64_t)m * g.ldd + n];
      if (g.tC) {
        float* c = static_cast<float*>(g.C) + ci;
        *c = g.epi == 2 ? *c + (float)(g.alpha * v) : (float)v;
      } else {
        double* c = static_cast<double*>(g.C) + ci;
        *c = g.epi == 2 ? *c + g.alpha * (double)v : (double)v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// a2 for small 2D patches (the coarse levels): the four contractions of one
// patch interior in one CTA, operands and intermediates in shared memory
// (row pitches odd, so that the strided operand reads hit distinct banks).
// A warp computes 4 rows x 128 columns (lane + 32 j) of a product per task.
// ---------------------------------------------------------------------------
template <typename T, typename FA, typename FB, typename FE>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, FA a_at, FB b_at, FE epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int mb = (M + 3) / 4, nbk = (N + 127) / 128;
  for (int t = warp; t < mb * nbk; t += nw) {
    const int m0 = (t / nbk) * 4, nb0 = (t % nbk) * 128 + lane;
    int mi[4], nj[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) mi[i] = min(m0 + i, M - 1);  // clamped: valid reads, results dropped
#pragma unroll
    for (int j = 0; j < 4; ++j) nj[j] = min(nb0 + 32 * j, N - 1);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int k = 0; k < K; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = a_at(mi[i], k);
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = b_at(k, nj[j]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (m0 + i < M && nb0 + 32 * j < N) epi(m0 + i, nb0 + 32 * j, acc[i][j]);
  }
}

__host__ __device__ constexpr int odd_pitch(int n) { return n | 1; }

template <typename T>
__global__ void __launch_bounds__(512) fd_small_2d(const FdSmall* __restrict__ patches, const double* __restrict__ r,
                                                   double* __restrict__ u, double tau) {
  extern __shared__ __align__(16) unsigned char fd_smem[];
  const FdSmall q = patches[blockIdx.x];
  const int n0 = q.n0, n1 = q.n1, N0 = q.N0;
  const int pu0 = odd_pitch(n0), pu1 = odd_pitch(n1), ps = odd_pitch(n0);
  T* U0 = reinterpret_cast<T*>(fd_smem);
  T* U1 = U0 + n0 * pu0;
  T* S1 = U1 + n1 * pu1;
  T* S2 = S1 + n1 * ps;
  const T* gU0 = static_cast<const T*>(q.U0);
  const T* gU1 = static_cast<const T*>(q.U1);
  const T* dinv = static_cast<const T*>(q.dinv);
  const double* rg = r + q.ibase;
  double* ug = u + q.ibase;
  for (int i = threadIdx.x; i < n0 * n0; i += blockDim.x) U0[(i / n0) * pu0 + i % n0] = gU0[i];
  for (int i = threadIdx.x; i < n1 * n1; i += blockDim.x) U1[(i / n1) * pu1 + i % n1] = gU1[i];
  for (int i = threadIdx.x; i < n1 * n0; i += blockDim.x) {
    const int i1 = i / n0, i0 = i % n0;
    S2[i1 * ps + i0] = (T)rg[(int64_t)i1 * N0 + i0];
  }
  __syncthreads();
  // 1) S1 = R U0
  cta_gemm<T>(n1, n0, n0, [&](int m, int k) { return S2[m * ps + k]; }, [&](int k, int n) { return U0[k * pu0 + n]; },
              [&](int m, int n, T v) { S1[m * ps + n] = v; });
  __syncthreads();
  // 2) S2 = (U1^T S1) * dinv
  cta_gemm<T>(n1, n0, n1, [&](int m, int k) { return U1[k * pu1 + m]; }, [&](int k, int n) { return S1[k * ps + n]; },
              [&](int m, int n, T v) { S2[m * ps + n] = v * dinv[m * n0 + n]; });
  __syncthreads();
  // 3) S1 = S2 U0^T
  cta_gemm<T>(n1, n0, n0, [&](int m, int k) { return S2[m * ps + k]; }, [&](int k, int n) { return U0[n * pu0 + k]; },
              [&](int m, int n, T v) { S1[m * ps + n] = v; });
  __syncthreads();
  // 4) u_interior += tau U1 S1
  cta_gemm<T>(n1, n0, n1, [&](int m, int k) { return U1[m * pu1 + k]; }, [&](int k, int n) { return S1[k * ps + n]; },
              [&](int m, int n, T v) { ug[(int64_t)m * N0 + n] += tau * (double)v; });
}

// ---------------------------------------------------------------------------
// a2 on the 5th-generation tensor cores: one 128 x 64 tile of a GemmTask per
// CTA (4 warps).  Operands are staged by all threads into shared memory in
// the K-major, non-swizzled core-matrix layout (8 rows x 16 bytes per core
// matrix; LBO = 128 B between core matrices along K, SBO = 1024 B between
// 8-row groups), converted to TF32 (kind::tf32) or BF16 (kind::f16) on the
// way; one thread issues tcgen05.mma (M = 128, N = 64, K = 32 bytes per
// instruction) into an FP32 accumulator in tensor memory, a commit to an
// mbarrier tells when the stage's buffer may be refilled (two buffers), and
// the epilogue reads the accumulator with tcgen05.ld (warp w: lanes 32w..).
// Every mbarrier wait is bounded; on expiry the CTA records the error,
// waits once more (bounded) for its MMAs and frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int UM = 128, UN = 64;   // tile, also the MMA shape
constexpr int UKB = 128;           // bytes of K per row per stage (4 MMAs of 32 bytes)
constexpr int kUmmaSmem = 2 * (UM + UN) * UKB;  // dynamic shared memory of gemm_umma

__device__ __forceinline__ uint64_t umma_sdesc(unsigned saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);           // start address
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;      // leading byte offset: next core matrix along K
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;     // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                            // descriptor version (tcgen05)
  return d;                                          // base offset 0, no swizzle
}

template <int KIND>
__device__ __forceinline__ unsigned umma_idesc() {
  // D = F32; A, B = TF32 (kind::tf32) or BF16 (kind::f16); both K-major;
  // N >> 3 at bit 17, M >> 4 at bit 24
  const unsigned ab = KIND == 0 ? 2u : 1u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((unsigned)(UN >> 3) << 17) | ((unsigned)(UM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void umma_store(unsigned char* tile, int row, int kk, float v) {
  // element kk of row `row` in the core-matrix layout of one stage
  constexpr int ES = KIND == 0 ? 4 : 2;
  const int byte = kk * ES;
  unsigned char* p = tile + (row >> 3) * 1024 + (byte >> 4) * 128 + (row & 7) * 16 + (byte & 15);
  if (KIND == 0) *reinterpret_cast<float*>(p) = v;
  else *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
}

template <int KIND>
__global__ void __launch_bounds__(128) gemm_umma(const GemmTask* __restrict__ tasks,
                                                 const GemmItem* __restrict__ items, int* err) {
  constexpr int ES = KIND == 0 ? 4 : 2;
  constexpr int KT = UKB / ES;  // K elements per stage
  // dynamic shared memory (kUmmaSmem bytes): two A and two B stage buffers
  extern __shared__ __align__(1024) unsigned char usm[];
  // stage buffer b: A at usm + b * UM * UKB, B at usm + 2 * UM * UKB + b * UN * UKB
  auto sA = [&](int b) { return usm + b * (UM * UKB); };
  auto sB = [&](int b) { return usm + 2 * UM * UKB + b * (UN * UKB); };
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ unsigned tmem_slot;
  const GemmItem it = items[blockIdx.x];
  const GemmTask g = tasks[it.task];
  const int64_t oA = it.z * g.sA, oB = it.z * g.sB, oC = it.z * g.sC;
  const int m0 = it.tm * UM, n0 = it.tn * UN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(UN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  const unsigned idesc = umma_idesc<KIND>();
  const int nst = (g.K + KT - 1) / KT;
  bool ok = true;
  unsigned phase_bits = 0;
  for (int st = 0; st < nst; ++st) {
    const int b = st & 1;
    if (st >= 2) {  // the MMAs that read this buffer two stages ago are done
      if (ok && !mbar_wait(smem_u32(&mbar[b]), (phase_bits >> b) & 1u)) {
        ok = false;
        atomicExch(err, 3);
      }
      phase_bits ^= 1u << b;
    }
    const int k0 = st * KT;
    // coalesced staging: consecutive threads read consecutive global addresses
    // (along k when it is the contiguous index, else along m / n)
#pragma unroll 4
    for (int i = 0; i < (UM * KT) / 128; ++i) {
      const int e = i * 128 + tid;
      const int row = g.transA ? e % UM : e / KT;
      const int kk = g.transA ? e / UM : e % KT;
      const int m = m0 + row, k = k0 + kk;
      float v = 0.0f;
      if (m < g.M && k < g.K)
        v = ldt<float>(g.A, oA + (g.transA ? (int64_t)k * g.lda + m : (int64_t)m * g.lda + k), g.tA);
      umma_store<KIND>(sA(b), row, kk, v);
    }
#pragma unroll 4
    for (int i = 0; i < (UN * KT) / 128; ++i) {
      const int e = i * 128 + tid;
      const int nr = g.transB ? e / KT : e % UN;
      const int kk = g.transB ? e % KT : e / UN;
      const int n = n0 + nr, k = k0 + kk;
      float v = 0.0f;
      if (n < g.N && k < g.K)
        v = ldt<float>(g.B, oB + (g.transB ? (int64_t)n * g.ldb + k : (int64_t)k * g.ldb + n), g.tB);
      umma_store<KIND>(sB(b), nr, kk, v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a0 = smem_u32(sA(b)), b0 = smem_u32(sB(b));
#pragma unroll
      for (int j = 0; j < UKB / 32; ++j) {
        const uint64_t ad = umma_sdesc(a0 + 256 * j), bd = umma_sdesc(b0 + 256 * j);
        const unsigned acc = (st > 0 || j > 0) ? 1u : 0u;
        if (KIND == 0)
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[b]))
                   : "memory");
    }
  }
  // wait for the last stage's commit (it covers every earlier MMA)
  if (nst > 0) {
    const int b = (nst - 1) & 1;
    if (!mbar_wait(smem_u32(&mbar[b]), (phase_bits >> b) & 1u)) {
      if (ok) atomicExch(err, 3);
      ok = false;
      mbar_wait(smem_u32(&mbar[b]), (phase_bits >> b) & 1u);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && nst > 0) {
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < UN; c0 += 16) {
      unsigned v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < g.M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = n0 + c0 + i;
          if (n >= g.N) continue;
          float acc = __uint_as_float(v[i]);
          const int64_t ci = oC + (int64_t)m * g.ldc + gcol(g, n);
          if (g.epi == 1) acc *= static_cast<const float*>(g.dinv)[(int64_t)m * g.ldd + n];
          if (g.tC) {
            float* c = static_cast<float*>(g.C) + ci;
            *c = g.epi == 2 ? *c + (float)(g.alpha * acc) : acc;
          } else {
            double* c = static_cast<double*>(g.C) + ci;
            *c = g.epi == 2 ? *c + g.alpha * (double)acc : (double)acc;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UN) : "memory");
}

// ---------------------------------------------------------------------------
// a2 on the tensor cores, TF32 with FP32 operands in memory: the same 128 x 64
// tile and core-matrix layout as gemm_umma, but the operands are copied
// element by element into shared memory by asynchronous copies (TF32 reads
// the FP32 bit patterns, so nothing passes through registers), through a ring
// of kUmmaStages slabs: the copies of slab s + 3 are in flight while the MMAs
// of slab s run.  A slab's buffer is refilled after the commit of the MMAs that
// read it has arrived on its mbarrier.  256 threads: all stage, thread 0
// issues the MMAs, the epilogue reads the accumulator with warp w taking TMEM
// lanes 32 (w mod 4).. and columns 32 (w / 4)...  Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int kUmmaStages = 4;
// core matrices of one 8-row group 144 B apart along K (not 128): the eight 16-byte copies that
// fill one row's slab then land in distinct shared-memory banks; 8-row groups 8 x 144 B apart
// K of one slab: 256 bytes per row (64 TF32 elements, 8 MMAs); a row's 16 core matrices along K
constexpr int kTfKB = 256;
constexpr int kTfLbo = 144, kTfSbo = (kTfKB / 16) * kTfLbo;
constexpr int kTfA = (UM / 8) * kTfSbo, kTfB = (UN / 8) * kTfSbo;  // bytes of one slab of A / B
constexpr int kUmmaTf32Smem = kUmmaStages * (kTfA + kTfB);

__device__ __forceinline__ uint64_t umma_sdesc_tf(unsigned saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);             // start address
  d |= (uint64_t)((kTfLbo >> 4) & 0x3FFFu) << 16;      // leading byte offset: next core matrix along K
  d |= (uint64_t)((kTfSbo >> 4) & 0x3FFFu) << 32;      // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                              // descriptor version (tcgen05)
  return d;                                            // base offset 0, no swizzle
}

__global__ void __launch_bounds__(256) gemm_umma_tf32(const GemmTask* __restrict__ tasks,
                                                      const GemmItem* __restrict__ items, int* err) {
  constexpr int KT = kTfKB / 4;  // K elements per slab
  extern __shared__ __align__(1024) unsigned char usm[];
  auto sA = [&](int b) { return usm + b * kTfA; };
  auto sB = [&](int b) { return usm + kUmmaStages * kTfA + b * kTfB; };
  __shared__ __align__(8) unsigned long long mbar[kUmmaStages];
  __shared__ unsigned tmem_slot;
  const GemmItem it = items[blockIdx.x];
  const GemmTask g = tasks[it.task];
  const float* Ag = static_cast<const float*>(g.A) + it.z * g.sA;
  const float* Bg = static_cast<const float*>(g.B) + it.z * g.sB;
  const int64_t oC = it.z * g.sC;
  const int m0 = it.tm * UM, n0 = it.tn * UN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(UN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < kUmmaStages; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  const unsigned idesc = umma_idesc<0>();
  const int nst = (g.K + KT - 1) / KT;
  const int64_t sAm = g.transA ? 1 : g.lda, sAk = g.transA ? g.lda : 1;
  const int64_t sBn = g.transB ? g.ldb : 1, sBk = g.transB ? 1 : g.ldb;
  // element (row, kk) of a slab in the core-matrix layout: 8-row groups kTfSbo B apart, 16-byte column groups
  auto cm_off = [](int row, int kk) {
    return (row >> 3) * kTfSbo + (kk >> 2) * kTfLbo + (row & 7) * 16 + (kk & 3) * 4;
  };
  auto load = [&](int st) {
    const int b = st % kUmmaStages, k0 = st * KT;
    unsigned char* a = sA(b);
    unsigned char* bb = sB(b);
    if (g.vec) {  // 16-byte copies: one core-matrix row segment (4 consecutive k) each
#pragma unroll
      for (int i = 0; i < (UM * KT / 4) / 256; ++i) {
        const int e = i * 256 + tid;
        const int row = e / (KT / 4), kq = e % (KT / 4);
        const int m = m0 + row, k = k0 + 4 * kq;
        const bool ok = m < g.M && k < g.K;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(a + cm_off(row, 4 * kq))),
                     "l"(ok ? Ag + (int64_t)m * g.lda + k : Ag), "r"(ok ? 16 : 0)
                     : "memory");
      }
#pragma unroll
      for (int i = 0; i < (UN * KT / 4) / 256; ++i) {
        const int e = i * 256 + tid;
        const int nr = e / (KT / 4), kq = e % (KT / 4);
        const int n = n0 + nr, k = k0 + 4 * kq;
        const bool ok = n < g.N && k < g.K;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(bb + cm_off(nr, 4 * kq))),
                     "l"(ok ? Bg + (int64_t)n * g.ldb + k : Bg), "r"(ok ? 16 : 0)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      return;
    }
#pragma unroll 4
    for (int i = 0; i < (UM * KT) / 256; ++i) {  // consecutive threads: consecutive global addresses
      const int e = i * 256 + tid;
      const int row = g.transA ? e % UM : e / KT, kk = g.transA ? e / UM : e % KT;
      const int m = m0 + row, k = k0 + kk;
      const bool ok = m < g.M && k < g.K;
      cp_async_elem<4>(a + cm_off(row, kk), ok ? Ag + m * sAm + k * sAk : Ag, ok);
    }
#pragma unroll 4
    for (int i = 0; i < (UN * KT) / 256; ++i) {
      const int e = i * 256 + tid;
      const int nr = g.transB ? e / KT : e % UN, kk = g.transB ? e % KT : e / UN;
      const int n = n0 + nr, k = k0 + kk;
      const bool ok = n < g.N && k < g.K;
      cp_async_elem<4>(bb + cm_off(nr, kk), ok ? Bg + n * sBn + k * sBk : Bg, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int st = 0; st < kUmmaStages - 1; ++st) {
    if (st < nst) load(st);
    else asm volatile("cp.async.commit_group;" ::: "memory");
  }
  bool ok = true;
  unsigned phase_bits = 0;
  for (int st = 0; st < nst; ++st) {
    const int b = st % kUmmaStages;
    asm volatile("cp.async.wait_group %0;" ::"n"(kUmmaStages - 2) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor cores
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a0 = smem_u32(sA(b)), b0 = smem_u32(sB(b));
#pragma unroll
      for (int j = 0; j < kTfKB / 32; ++j) {
        const uint64_t ad = umma_sdesc_tf(a0 + 2 * kTfLbo * j), bd = umma_sdesc_tf(b0 + 2 * kTfLbo * j);
        const unsigned acc = (st > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[b]))
                   : "memory");
    }
    // refill the buffer of slab st - 1 once its MMAs are done
    const int nxt = st + kUmmaStages - 1;
    if (nxt < nst) {
      if (st >= 1) {
        const int pb = (st - 1) % kUmmaStages;
        if (ok && !mbar_wait(smem_u32(&mbar[pb]), (phase_bits >> pb) & 1u)) {
          ok = false;
          atomicExch(err, 3);
        }
        phase_bits ^= 1u << pb;
      }
      load(nxt);
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // the commits of the last slabs were not consumed in the loop: wait for them in order (slab t is
  // use t / kUmmaStages of its buffer; every earlier use of that buffer has been waited for)
  for (int t = max(0, nst - kUmmaStages); t < nst; ++t) {
    const int tb = t % kUmmaStages;
    const unsigned par = (unsigned)((t / kUmmaStages) & 1);
    if (!mbar_wait(smem_u32(&mbar[tb]), par)) {
      if (ok) atomicExch(err, 3);
      ok = false;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: accumulator -> shared memory (the stage buffers are free: every MMA has completed and
  // every copy has landed) -> global memory with consecutive threads on consecutive addresses
  constexpr int TP = UN + 1;  // tile pitch in floats (odd: conflict-free column reads)
  float* tile = reinterpret_cast<float*>(usm);
  __syncthreads();
  if (ok && nst > 0) {
    const int q = warp & 3, h = warp >> 2;
    const int row = q * 32 + lane;
#pragma unroll
    for (int c0 = h * 32; c0 < h * 32 + 32; c0 += 16) {
      unsigned v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) tile[row * TP + c0 + i] = __uint_as_float(v[i]);
    }
  }
  __syncthreads();
  if (ok && nst > 0) {
    for (int idx = tid; idx < UM * UN; idx += 256) {
      const int r = g.ctrans ? idx % UM : idx / UN, c = g.ctrans ? idx / UM : idx % UN;
      const int m = m0 + r, n = n0 + c;
      if (m >= g.M || n >= g.N) continue;
      float acc = tile[r * TP + c];
      const int64_t ci = oC + (g.ctrans ? (int64_t)n * g.ldc + m : (int64_t)m * g.ldc + gcol(g, n));
      if (g.epi == 1) acc *= static_cast<const float*>(g.dinv)[(int64_t)m * g.ldd + n];
      if (g.tC) {
        float* cp = static_cast<float*>(g.C) + ci;
        *cp = g.epi == 2 ? *cp + (float)(g.alpha * acc) : acc;
      } else {
        double* cp = static_cast<double*>(g.C) + ci;
        *cp = g.epi == 2 ? *cp + g.alpha * (double)acc : (double)acc;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UN) : "memory");
}

// the interiors of all patches of r as compact FP32 blocks: patch k's row i1 of n0 values at
// dst + d_off[k] + i1 * d_ld[k] (the padding columns stay 0); one thread per element
__global__ void gather_interior_f32(int npatch, const int64_t* __restrict__ e_ptr, const int64_t* __restrict__ ibase,
                                    const int* __restrict__ n0s, const int* __restrict__ N0s,
                                    const int64_t* __restrict__ d_off, const int* __restrict__ d_ld,
                                    const double* __restrict__ r, float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= e_ptr[npatch]) return;
  int k = 0;
  while (e >= e_ptr[k + 1]) ++k;  // few patches
  const int64_t loc = e - e_ptr[k];
  const int n0 = n0s[k];
  const int64_t i1 = loc / n0, i0 = loc % n0;
  dst[d_off[k] + i1 * d_ld[k] + i0] = (float)r[ibase[k] + i1 * N0s[k] + i0];
}

// FP64 -> FP32 copy of a vector (the residual for the tensor-core contractions)
__global__ void to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

// ---------------------------------------------------------------------------
// a3 / a7: dense solves with precomputed inverses, z = Z r_T, u_T += tau z
// (mode 0) or u_T = z (mode 1).  T: element type of Z and of the arithmetic
// (double; float for the interface pieces of the mixed-precision smoother).
// ---------------------------------------------------------------------------
constexpr int kPieceRows = 64;

template <typename T>
__global__ void __launch_bounds__(256) piece_apply(const PieceItem* __restrict__ items,
                                                   const PieceMeta* __restrict__ pieces,
                                                   const T* __restrict__ zpool,
                                                   const int64_t* __restrict__ piece_pos,
                                                   const double* __restrict__ r, double* __restrict__ u,
                                                   double tau, int mode) {
  extern __shared__ __align__(16) unsigned char piece_smem[];
  T* rs = reinterpret_cast<T*>(piece_smem);
  const PieceItem it = items[blockIdx.x];
  const PieceMeta pm = pieces[it.piece];
  const int64_t* pp = piece_pos + pm.dof_off;
  for (int i = threadIdx.x; i < pm.n; i += blockDim.x) rs[i] = (T)r[pp[i]];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rend = min(pm.n, it.row0 + kPieceRows);
  for (int row = it.row0 + warp; row < rend; row += 8) {
    const T* z = zpool + pm.z_off + (int64_t)row * pm.n;
    T s = 0;
    for (int j = lane; j < pm.n; j += 32) s = fma(z[j], rs[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (mode == 0) u[pp[row]] += tau * (double)s;
      else u[pp[row]] = (double)s;
    }
  }
}

// ---------------------------------------------------------------------------
// a4 (sweep): all colours of one sweep in a single cooperative launch.
// Rows of a colour are spread over the whole grid, TPR lanes per row (each
// lane sums a share of the (2p+1)^d stencil, then a shuffle reduction); the
// coefficients come from a copy of the band in colour order, so consecutive
// rows of a colour read consecutive addresses.  A grid barrier separates the
// colours; it gives up after a bounded wait and reports it in *err.
// u and f are read through L2 (ld.cg): other SMs wrote them since the last
// barrier and L1 is not coherent.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* err) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (++spins > (1ll << 22)) {  // ~0.3-1 s: a co-resident grid never waits this long
          atomicExch(err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)err) == 0;
}

// One Gauss-Seidel row update for each row group of TPR lanes of a warp:
// rows base + lane / TPR (those below e1).  Each lane sums a share of the
// (2p+1)^d stencil and of the SIPG couplings, the group reduces by shuffles
// and its first lane writes u_i + (f_i - sum_j a_ij u_j) / a_ii.
// TB: type of the colour-ordered coefficients and of the arithmetic (double
// for the FP64 path, float for the mixed path); u and f stay FP64 and are
// read through L2 (ld.cg): other SMs wrote them since the last barrier.
template <int D, int P, int TPR, typename TB>
__device__ __forceinline__ void gs_rows(const GsSweepArgs& a, int64_t base, int64_t e1) {
  constexpr int W = 2 * P + 1;
  constexpr int NOB = D == 2 ? W : W * W;  // offset blocks of W consecutive o0
  constexpr int center = D == 2 ? P * W + P : (P * W + P) * W + P;
  const TB* gsband = static_cast<const TB*>(a.gsband);
  const int lane = threadIdx.x & 31;
  const int sub = lane % TPR;
  const int64_t e = base + lane / TPR;
  const bool active = e < e1;
  TB acc = 0;
  int64_t pos = 0;
  double upos = 0.0, fpos = 0.0;
  TB diag = 1;
  int cls = -1;
  if (active) {
    // independent loads first: position, strides, couplings, diagonal, u_i, f_i
    pos = a.gs_pos[e];
    const int2 st = a.gs_stride[e];
    const int2 xr = a.gs_xrange[e];
    cls = a.gs_cls[e];
    diag = __ldg(gsband + (int64_t)center * a.ngs + e);
    upos = __ldcg(a.u + pos);
    fpos = __ldcg(a.f + pos);
    const int64_t s1 = st.x, s2 = st.y;
    for (int ob = sub; ob < NOB; ob += TPR) {
      const int o1 = ob % W, o2 = ob / W;
      const int64_t off = (D == 3 ? (int64_t)(o2 - P) * s2 : 0) + (int64_t)(o1 - P) * s1 - P;
      const TB* br = gsband + (int64_t)ob * W * a.ngs + e;
      const double* ur = a.u + pos + off;
#pragma unroll
      for (int o0 = 0; o0 < W; ++o0) acc = fma(__ldg(br + (int64_t)o0 * a.ngs), (TB)__ldcg(ur + o0), acc);
    }
    // SIPG couplings across interfaces and, for a DoF shared by conforming patches, the band rows
    // of its further copies (their diagonals are part of the entry's), shared over the row's lanes;
    // four entries per lane in flight (the column then the value: two dependent loads each), summed
    // in the same order as one at a time
    int j = xr.x + sub;
    for (; j + 3 * TPR < xr.y; j += 4 * TPR) {
      int64_t c[4];
      double v[4], w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        c[q] = a.x_col[j + q * TPR];
        v[q] = a.x_val[j + q * TPR];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = __ldcg(a.u + c[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = fma((TB)v[q], (TB)w[q], acc);
    }
    for (; j < xr.y; j += TPR) acc = fma((TB)a.x_val[j], (TB)__ldcg(a.u + a.x_col[j]), acc);
  }
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (active && sub == 0) {
    const double unew = upos + (double)(((TB)fpos - acc) / diag);
    if (cls < 0) {
      a.u[pos] = unew;
    } else {
      for (int cp = a.sh_ptr[cls]; cp < a.sh_ptr[cls + 1]; ++cp) a.u[a.sh_pos[cp]] = unew;
    }
  }
}

// Colours [c_begin, c_end) of a sweep over the whole grid, one cooperative
// launch, a bounded grid barrier between colours (used for the colours that
// couple patches of one parity).
template <int D, int P, int TPR, typename TB>
__global__ void __launch_bounds__(256) gs_sweep_coop(GsSweepArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp_global = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t rows_per_warp = 32 / TPR;
  const int64_t rows_per_grid = ((int64_t)gridDim.x * blockDim.x) / TPR;
  (void)lane;
  const int nc = a.c_end - a.c_begin;
  for (int ci = 0; ci < nc; ++ci) {
    const int c = a.forward ? a.c_begin + ci : a.c_end - 1 - ci;
    const int e0 = a.cptr[c], e1 = a.cptr[c + 1];
    for (int64_t base = e0 + warp_global * rows_per_warp; base < e1; base += rows_per_grid)
      gs_rows<D, P, TPR, TB>(a, base, e1);
    if (gridDim.x == 1) {
      __syncthreads();  // one block: its own writes are visible after the barrier
    } else if (!grid_barrier(a.bar, a.err)) {
      return;
    }
  }
}

// f minus the couplings to the other parity (SIPG cross-patch terms, from the
// current u) for the base-colour entries [e0, e0 + n) of one phase, into their
// blocks: entries without such terms one thread each (the first n threads),
// the nx entries with them (xent) one warp each, lanes over the couplings
__global__ void gs_fill_phase(int e0, int n, int nx, const int* __restrict__ xent, const int64_t* __restrict__ f_off,
                              const int64_t* __restrict__ gs_pos, const int2* __restrict__ xrange,
                              const int64_t* __restrict__ x_col, const double* __restrict__ x_val,
                              const double* __restrict__ f, const double* __restrict__ u, unsigned char* pool) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncopy = ((int64_t)n + 31) / 32 * 32;
  if (tid < ncopy) {
    if (tid >= n) return;
    const int e = e0 + (int)tid;
    const int64_t o = f_off[e];
    const int2 xr = xrange[e];
    if (o < 0 || xr.y > xr.x) return;  // entries with couplings: their warp below
    *reinterpret_cast<float*>(pool + o) = (float)f[gs_pos[e]];
    return;
  }
  const int64_t w = (tid - ncopy) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nx) return;
  const int e = xent[w];
  const int2 xr = xrange[e];
  double v = 0.0;
  for (int j = xr.x + lane; j < xr.y; j += 32) v += x_val[j] * u[x_col[j]];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int64_t o = f_off[e];
  if (lane == 0 && o >= 0) *reinterpret_cast<float*>(pool + o) = (float)(f[gs_pos[e]] - v);
}

// ---------------------------------------------------------------------------
// a8: PCG vectors and deterministic reductions
// ---------------------------------------------------------------------------
constexpr int kRedBlocks = 304;  // 2 x 152 SMs; fixed so the reduction order is fixed

// block sum into partials[blockIdx]; the last block to finish (ticket taken
// from *counter, which it resets) sums the partials in a fixed order and
// applies `op` to the scalar slots
__device__ void finish_reduction(double v, double* partials, double* scal, int op, int slot,
                                 unsigned int* counter) {
  __shared__ double sh[32];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += sh[i];
    partials[blockIdx.x] = b;
    __threadfence();
    const unsigned int done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  if (threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (int i = 0; i < (int)gridDim.x; ++i) tot += ((volatile double*)partials)[i];
    scal[slot] = tot;
    if (op == 1) scal[S_ALPHA] = scal[S_RZ] / tot;                         // slot = S_PQ
    if (op == 2) { scal[S_BETA] = tot / scal[S_RZ]; scal[S_RZ] = tot; }    // slot = S_RZNEW
    // flexible CG (Polak-Ribiere): beta = r.(z_new - z_old) / (r_old . z_old)
    if (op == 3) { scal[S_BETA] = (tot - scal[S_RZOLD]) / scal[S_RZ]; scal[S_RZ] = tot; }
    *counter = 0u;
  }
}

// scal[slot] = sum_i w_i a_i b_i  (w may be null)
__global__ void __launch_bounds__(256) dot_kernel(int64_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, const double* __restrict__ w,
                                                  double* partials, double* scal, unsigned int* counter,
                                                  int slot, int op) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[i] * b[i];
    s += w ? w[i] * v : v;
  }
  finish_reduction(s, partials, scal, op, slot, counter);
}

// x += alpha p; r -= alpha q; scal[S_RR] = sum w r^2
__global__ void __launch_bounds__(256) cg_update_xr(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    const double* __restrict__ w, double* partials,
                                                    double* scal, unsigned int* counter) {
  const double alpha = scal[S_ALPHA];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s += w ? w[i] * ri * ri : ri * ri;
  }
  finish_reduction(s, partials, scal, 0, S_RR, counter);
}

// p = z + beta p
__global__ void cg_update_p(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                            const double* __restrict__ scal) {
  const double beta = scal[S_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// Device-side control of the PCG loop (Sec. 4, the stopping rule with the recursive residual,
// confirmed by the true one), one thread, after the first half of an iteration: records the
// relative residual, and sets the conditions of the graph's loop (hloop), of the true-residual
// confirmation (hconf) and of the second half of the iteration (hcont)
__global__ void cg_ctl_a(const double* __restrict__ scal, CgLoopState* st, double* hist,
                         cudaGraphConditionalHandle hloop, cudaGraphConditionalHandle hconf,
                         cudaGraphConditionalHandle hcont) {
  const int it = ++st->it;
  const double pq = scal[S_PQ];
  const double rel = sqrt(scal[S_RR]) / scal[S_NF];
  hist[it] = rel;
  st->rel = rel;
  if (!(pq > 0.0) || !isfinite(rel)) {
    st->status = 3;
    cudaGraphSetConditional(hloop, 0);
    cudaGraphSetConditional(hconf, 0);
    cudaGraphSetConditional(hcont, 0);
    return;
  }
  if (rel <= scal[S_TOL]) {
    st->nconf++;
    cudaGraphSetConditional(hconf, 1);
    cudaGraphSetConditional(hcont, 0);  // decided by cg_ctl_c
    return;
  }
  cudaGraphSetConditional(hconf, 0);
  if (it >= (int)scal[S_MAXIT]) {
    st->status = 2;
    cudaGraphSetConditional(hloop, 0);
    cudaGraphSetConditional(hcont, 0);
  } else {
    st->ncont++;
    cudaGraphSetConditional(hcont, 1);
  }
}

// after the confirming true residual ||f - A x||^2 in scal[S_TMP]
__global__ void cg_ctl_c(const double* __restrict__ scal, CgLoopState* st, double* hist,
                         cudaGraphConditionalHandle hloop, cudaGraphConditionalHandle hcont) {
  const double trel = sqrt(scal[S_TMP]) / scal[S_NF];
  if (trel <= scal[S_TOL]) {  // the history ends with the confirmed (true) residual
    hist[st->it] = trel;
    st->rel = trel;
    st->status = 1;
    cudaGraphSetConditional(hloop, 0);
    cudaGraphSetConditional(hcont, 0);
  } else if (st->it >= (int)scal[S_MAXIT]) {
    st->status = 2;
    cudaGraphSetConditional(hloop, 0);
    cudaGraphSetConditional(hcont, 0);
  } else {
    st->ncont++;
    cudaGraphSetConditional(hcont, 1);
  }
}

// before the loop of a solve that runs as one graph: ||f||^2 in scal[S_FF], ||f - A u0||^2 in
// scal[S_RR]; decides between a non-finite input (status 4), a zero right-hand side (status 5, the
// solution is zero: hzero), an initial guess that meets the rule (status 1), the iteration limit 0
// (status 2) and the iteration (hgo: the first cycle; hloop: the loop)
__global__ void cg_ctl_0(double* scal, CgLoopState* st, double* hist, cudaGraphConditionalHandle hzero,
                         cudaGraphConditionalHandle hgo, cudaGraphConditionalHandle hloop) {
  const double ff = scal[S_FF], rr = scal[S_RR];
  cudaGraphSetConditional(hzero, 0);
  cudaGraphSetConditional(hgo, 0);
  cudaGraphSetConditional(hloop, 0);
  if (!isfinite(ff) || !isfinite(rr)) {
    st->status = 4;
    return;
  }
  if (!(ff > 0.0)) {
    st->status = 5;
    st->rel = 0.0;
    hist[0] = 0.0;
    cudaGraphSetConditional(hzero, 1);
    return;
  }
  const double nf = sqrt(ff);
  scal[S_NF] = nf;
  const double rel = sqrt(rr) / nf;
  hist[0] = rel;
  st->rel = rel;
  if (rel <= scal[S_TOL]) {
    st->status = 1;
    return;
  }
  if ((int)scal[S_MAXIT] <= 0) {
    st->status = 2;
    return;
  }
  cudaGraphSetConditional(hgo, 1);
  cudaGraphSetConditional(hloop, 1);
}

__global__ void cg_loop_init(double* scal, CgLoopState* st, double tol, double nf, int maxit) {
  scal[S_TOL] = tol;
  if (nf > 0.0) scal[S_NF] = nf;
  scal[S_MAXIT] = (double)maxit;
  st->it = 0;
  st->status = 0;
  st->nconf = 0;
  st->ncont = 0;
  st->rel = 0.0;
}

__global__ void scatter_global(int64_t nloc, const int* __restrict__ l2g, const double* __restrict__ g,
                               double* __restrict__ loc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nloc; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = l2g[i];
    loc[i] = k >= 0 ? g[k] : 0.0;
  }
}

__global__ void gather_global(int ndof, const int64_t* __restrict__ owner, const double* __restrict__ loc,
                              double* __restrict__ g) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += gridDim.x * blockDim.x) g[i] = loc[owner[i]];
}

// y = x + s * z  (element-wise), used for u += e and copies
__global__ void axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

// ---------------------------------------------------------------------------
// launchers (each counts the kernels it enqueues)
// ---------------------------------------------------------------------------
static thread_local long long g_launches = 0;
long long launch_counter() { return g_launches; }
void count_launch() { ++g_launches; }
template <int D, int MODE>
static void launch_band_p(int p, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pm,
                          const double* band, int64_t nloc, const double* u, const double* f, double* out) {
  switch (p) {
#define MG_CASE(PP) \
  case PP: band_apply<D, PP, MODE><<<ntiles, kTile, 0, st>>>(tiles, pm, band, nloc, u, f, out); break;
    MG_CASE(1) MG_CASE(2) MG_CASE(3) MG_CASE(4) MG_CASE(5) MG_CASE(6) MG_CASE(7) MG_CASE(8)
#undef MG_CASE
    default: break;
  }
}

void launch_band(int d, int p, int mode, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pm,
                 const double* band, int64_t nloc, const double* u, const double* f, double* out) {
  if (ntiles == 0) return;
  ++g_launches;
  if (d == 2) {
    if (mode == 0) launch_band_p<2, 0>(p, ntiles, st, tiles, pm, band, nloc, u, f, out);
    else launch_band_p<2, 1>(p, ntiles, st, tiles, pm, band, nloc, u, f, out);
  } else {
    if (mode == 0) launch_band_p<3, 0>(p, ntiles, st, tiles, pm, band, nloc, u, f, out);
    else launch_band_p<3, 1>(p, ntiles, st, tiles, pm, band, nloc, u, f, out);
  }
}

void launch_band_residual_f32(int d, int p, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pm,
                              const float* band32, int64_t nloc, const double* u, const double* f, double* out,
                              int g) {
  if (ntiles == 0) return;
  ++g_launches;
  // g threads per row group; 0: four unless the level alone fills the GPU with one
  if (g != 1 && g != 2 && g != 4) g = nloc < 400000 ? 4 : 1;
  constexpr int NG = kTile / kRowsF32;
  switch (p) {
#define MG_LAUNCH(DD, PP, GG) \
  band_residual_f32<DD, PP, GG><<<ntiles, NG * GG, 0, st>>>(tiles, pm, band32, nloc, u, f, out)
#define MG_CASE(PP)                                                                              \
  case PP:                                                                                       \
    if (d == 2) {                                                                                \
      if (g == 4) MG_LAUNCH(2, PP, 4); else if (g == 2) MG_LAUNCH(2, PP, 2); else MG_LAUNCH(2, PP, 1); \
    } else {                                                                                     \
      if (g == 4) MG_LAUNCH(3, PP, 4); else if (g == 2) MG_LAUNCH(3, PP, 2); else MG_LAUNCH(3, PP, 1); \
    }                                                                                            \
    break;
    MG_CASE(1) MG_CASE(2) MG_CASE(3) MG_CASE(4) MG_CASE(5) MG_CASE(6) MG_CASE(7) MG_CASE(8)
#undef MG_CASE
#undef MG_LAUNCH
    default: break;
  }
}

void launch_cross(int mode, int nx, cudaStream_t st, const int64_t* x_row, const int* x_ptr, const int64_t* x_col,
                  const double* x_val, const double* u, double* out) {
  if (nx == 0) return;
  const int blocks = (nx * 32 + 255) / 256;
  ++g_launches;
  if (mode == 0) cross_apply<0><<<blocks, 256, 0, st>>>(nx, x_row, x_ptr, x_col, x_val, u, out);
  else cross_apply<1><<<blocks, 256, 0, st>>>(nx, x_row, x_ptr, x_col, x_val, u, out);
}

void launch_shared(int nsh, cudaStream_t st, const int* sh_ptr, const int64_t* sh_pos, double* v, const double* f,
                   int mode) {
  if (nsh == 0) return;
  ++g_launches;
  shared_reduce<<<(nsh + 255) / 256, 256, 0, st>>>(nsh, sh_ptr, sh_pos, v, f, mode);
}

void launch_restrict(int d, bool f32, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pc,
                     const PatchMeta* pf, const XferMeta* xm, const int* ch_start, const double* ch_val, int cw,
                     const double* r, const double* w, const int* c_l2g, double* out) {
  if (ntiles == 0) return;
  ++g_launches;
#define MG_RESTRICT(DD, TT) \
  restrict_band<DD, TT><<<ntiles, kTile, 0, st>>>(tiles, pc, pf, xm, ch_start, ch_val, cw, r, w, c_l2g, out)
  if (d == 2) {
    if (f32) MG_RESTRICT(2, float); else MG_RESTRICT(2, double);
  } else {
    if (f32) MG_RESTRICT(3, float); else MG_RESTRICT(3, double);
  }
#undef MG_RESTRICT
}

void launch_prolong(int d, bool f32, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pf,
                    const PatchMeta* pc, const XferMeta* xm, const int* par_start, const double* par_val, int pw,
                    const double* e, double* u) {
  if (ntiles == 0) return;
  ++g_launches;
#define MG_PROLONG(DD, TT) \
  prolong_band<DD, TT><<<ntiles, kTile, 0, st>>>(tiles, pf, pc, xm, par_start, par_val, pw, e, u)
  if (d == 2) {
    if (f32) MG_PROLONG(2, float); else MG_PROLONG(2, double);
  } else {
    if (f32) MG_PROLONG(3, float); else MG_PROLONG(3, double);
  }
#undef MG_PROLONG
}

void launch_restrict_mw2(bool f32, int nblocks, int smem, cudaStream_t st, const int4* blocks, const PatchMeta* pc,
                         const PatchMeta* pf, const XferMeta* xm, const int* ch_start, const double* ch_val, int cw,
                         const double* r, const double* w, const int* c_l2g, double* out) {
  if (nblocks == 0) return;
  ++g_launches;
  if (f32) restrict_mw2<float><<<nblocks, 256, smem, st>>>(blocks, pc, pf, xm, ch_start, ch_val, cw, r, w, c_l2g, out);
  else restrict_mw2<double><<<nblocks, 256, smem, st>>>(blocks, pc, pf, xm, ch_start, ch_val, cw, r, w, c_l2g, out);
}

void launch_prolong_mw2(bool f32, int nblocks, int smem, cudaStream_t st, const int4* blocks, const PatchMeta* pf,
                        const PatchMeta* pc, const XferMeta* xm, const int* par_start, const double* par_val, int pw,
                        const double* e, double* u) {
  if (nblocks == 0) return;
  ++g_launches;
  if (f32) prolong_mw2<float><<<nblocks, 256, smem, st>>>(blocks, pf, pc, xm, par_start, par_val, pw, e, u);
  else prolong_mw2<double><<<nblocks, 256, smem, st>>>(blocks, pf, pc, xm, par_start, par_val, pw, e, u);
}

cudaError_t prepare_transfers_mw2() {
  for (cudaError_t e : {cudaFuncSetAttribute(restrict_mw2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kXferSmemMax),
                        cudaFuncSetAttribute(restrict_mw2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kXferSmemMax),
                        cudaFuncSetAttribute(prolong_mw2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kXferSmemMax),
                        cudaFuncSetAttribute(prolong_mw2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kXferSmemMax)})
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

int gemm_tile(int arith) { return arith == 1 ? 64 : 32; }

int fd_small_smem(int n0, int n1, bool f32) {
  const size_t e = f32 ? sizeof(float) : sizeof(double);
  return (int)(e * ((size_t)n0 * odd_pitch(n0) + (size_t)n1 * odd_pitch(n1) + 2 * (size_t)n1 * odd_pitch(n0)));
}

cudaError_t prepare_fd_small() {
  cudaError_t e = cudaFuncSetAttribute(fd_small_2d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFdSmallSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fd_small_2d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFdSmallSmem);
}

void launch_fd_small(int npatch, int smem, bool f32, cudaStream_t st, const FdSmall* patches, const double* r,
                     double* u, double tau) {
  if (npatch == 0) return;
  ++g_launches;
  if (f32) fd_small_2d<float><<<npatch, 512, smem, st>>>(patches, r, u, tau);
  else fd_small_2d<double><<<npatch, 512, smem, st>>>(patches, r, u, tau);
}

void launch_gemm_umma(int nitems, int kind, cudaStream_t st, const GemmTask* tasks, const GemmItem* items, int* err) {
  if (nitems == 0) return;
  ++g_launches;
  if (kind == 0) gemm_umma<0><<<nitems, 128, kUmmaSmem, st>>>(tasks, items, err);
  else gemm_umma<1><<<nitems, 128, kUmmaSmem, st>>>(tasks, items, err);
}

cudaError_t prepare_gemm_umma() {
  cudaError_t e = cudaFuncSetAttribute(gemm_umma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gemm_umma_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaTf32Smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(gemm_umma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem);
}

void launch_gemm_umma_tf32(int nitems, cudaStream_t st, const GemmTask* tasks, const GemmItem* items, int* err) {
  if (nitems == 0) return;
  ++g_launches;
  gemm_umma_tf32<<<nitems, 256, kUmmaTf32Smem, st>>>(tasks, items, err);
}

void launch_gather_interior_f32(int npatch, int64_t total, cudaStream_t st, const int64_t* e_ptr,
                                const int64_t* ibase, const int* n0s, const int* N0s, const int64_t* d_off,
                                const int* d_ld, const double* r, float* dst) {
  if (total <= 0) return;
  ++g_launches;
  gather_interior_f32<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(npatch, e_ptr, ibase, n0s, N0s, d_off, d_ld,
                                                                       r, dst);
}

void launch_to_f32(int64_t n, cudaStream_t st, const double* x, float* y) {
  if (n <= 0) return;
  ++g_launches;
  to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y);
}

using GemmF64 = GemmSmem<32, double, double, double, kGemmStagesF64>;
using GemmF32A64 = GemmSmem<64, float, double, float, kGemmStagesF32>;
using GemmF32 = GemmSmem<64, float, float, float, kGemmStagesF32>;

cudaError_t prepare_gemm() {
  cudaError_t e = cudaFuncSetAttribute(gemm_tiled<64, float, double, float, kGemmStagesF32>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GemmF32A64::bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gemm_tiled<64, float, float, float, kGemmStagesF32>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GemmF32::bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(gemm_tiled<32, double, double, double, kGemmStagesF64>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GemmF64::bytes);
}

void launch_gemm(int nitems, int arith, int tA, cudaStream_t st, const GemmTask* tasks, const GemmItem* items) {
  if (nitems <= 0) return;
  ++g_launches;
  if (arith == 1) {
    if (tA == 0)
      gemm_tiled<64, float, double, float, kGemmStagesF32><<<nitems, 256, GemmF32A64::bytes, st>>>(tasks, items);
    else
      gemm_tiled<64, float, float, float, kGemmStagesF32><<<nitems, 256, GemmF32::bytes, st>>>(tasks, items);
  } else {
    gemm_tiled<32, double, double, double, kGemmStagesF64><<<nitems, 256, GemmF64::bytes, st>>>(tasks, items);
  }
}

template <int D, int P>
static void* gs_coop_func(bool f32) {
  return f32 ? (void*)gs_sweep_coop<D, P, 8, float> : (void*)gs_sweep_coop<D, P, 8, double>;
}

static void* gs_coop_ptr(int d, int p, bool f32) {
  switch (p) {
#define MG_CASE(PP) \
  case PP: return d == 2 ? gs_coop_func<2, PP>(f32) : gs_coop_func<3, PP>(f32);
    MG_CASE(1) MG_CASE(2) MG_CASE(3) MG_CASE(4) MG_CASE(5) MG_CASE(6) MG_CASE(7) MG_CASE(8)
#undef MG_CASE
    default: return nullptr;
  }
}

int gs_coop_max_blocks(int d, int p, bool f32) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs_coop_ptr(d, p, f32), 256, 0) != cudaSuccess)
    return 0;
  return sms * per_sm;
}

cudaError_t launch_gs_sweep(int d, int p, bool f32, int blocks, cudaStream_t st, GsSweepArgs a) {
  ++g_launches;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(gs_coop_ptr(d, p, f32), dim3(blocks), dim3(256), args, 0, st);
}

// One thread waits, with the kernels' bounded-wait routine and `limit` polls,
// on an mbarrier phase that nothing completes, and records the expiry in
// *err the way the kernels do (no copy or peer is involved, so nothing is
// left in flight); *elapsed_ns: the wait's duration by the global timer.
__global__ void wait_expiry_probe(long long limit, int* err, long long* elapsed_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
  unsigned long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  const bool done = mbar_wait(smem_u32(&bar), 0u, limit);
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  *elapsed_ns = (long long)(t1 - t0);
  if (!done) atomicExch(err, 2);
}

void launch_wait_expiry_probe(long long limit, cudaStream_t st, int* err, long long* elapsed_ns) {
  ++g_launches;
  wait_expiry_probe<<<1, 32, 0, st>>>(limit, err, elapsed_ns);
}

void launch_gs_fill_phase(int e0, int n, int nx, const int* xent, cudaStream_t st, const int64_t* f_off,
                          const int64_t* gs_pos, const int2* xrange, const int64_t* x_col, const double* x_val,
                          const double* f, const double* u, unsigned char* pool) {
  if (n <= 0) return;
  ++g_launches;
  const int64_t threads = ((int64_t)n + 31) / 32 * 32 + 32 * (int64_t)nx;
  gs_fill_phase<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(e0, n, nx, xent, f_off, gs_pos, xrange, x_col,
                                                                  x_val, f, u, pool);
}

void launch_piece(int nitems, int max_n, cudaStream_t st, const PieceItem* items, const PieceMeta* pieces,
                  const void* zpool, bool zf32, const int64_t* piece_pos, const double* r, double* u, double tau,
                  int mode) {
  if (nitems == 0) return;
  ++g_launches;
  if (zf32)
    piece_apply<float><<<nitems, 256, (size_t)max_n * sizeof(float), st>>>(
        items, pieces, static_cast<const float*>(zpool), piece_pos, r, u, tau, mode);
  else
    piece_apply<double><<<nitems, 256, (size_t)max_n * sizeof(double), st>>>(
        items, pieces, static_cast<const double*>(zpool), piece_pos, r, u, tau, mode);
}

cudaError_t prepare_piece_kernel(int max_n) {
  const size_t bytes = (size_t)max_n * sizeof(double);
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(piece_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(piece_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  return cudaSuccess;
}

void launch_dot(int64_t n, cudaStream_t st, const double* a, const double* b, const double* w, double* partials,
                double* scal, unsigned int* counter, int slot, int op) {
  ++g_launches;
  dot_kernel<<<kRedBlocks, 256, 0, st>>>(n, a, b, w, partials, scal, counter, slot, op);
}

void launch_cg_xr(int64_t n, cudaStream_t st, double* x, double* r, const double* p, const double* q,
                  const double* w, double* partials, double* scal, unsigned int* counter) {
  ++g_launches;
  cg_update_xr<<<kRedBlocks, 256, 0, st>>>(n, x, r, p, q, w, partials, scal, counter);
}

void launch_cg_ctl_a(cudaStream_t st, const double* scal, CgLoopState* state, double* hist,
                     unsigned long long hloop, unsigned long long hconf, unsigned long long hcont) {
  ++g_launches;
  cg_ctl_a<<<1, 1, 0, st>>>(scal, state, hist, hloop, hconf, hcont);
}

void launch_cg_ctl_c(cudaStream_t st, const double* scal, CgLoopState* state, double* hist,
                     unsigned long long hloop, unsigned long long hcont) {
  ++g_launches;
  cg_ctl_c<<<1, 1, 0, st>>>(scal, state, hist, hloop, hcont);
}

void launch_cg_ctl_0(cudaStream_t st, double* scal, CgLoopState* state, double* hist, unsigned long long hzero,
                     unsigned long long hgo, unsigned long long hloop) {
  ++g_launches;
  cg_ctl_0<<<1, 1, 0, st>>>(scal, state, hist, hzero, hgo, hloop);
}

void launch_cg_loop_init(cudaStream_t st, double* scal, CgLoopState* state, double tol, double nf, int maxit) {
  ++g_launches;
  cg_loop_init<<<1, 1, 0, st>>>(scal, state, tol, nf, maxit);
}

void launch_cg_p(int64_t n, cudaStream_t st, double* p, const double* z, const double* scal) {
  ++g_launches;
  cg_update_p<<<kRedBlocks * 2, 256, 0, st>>>(n, p, z, scal);
}

void launch_scatter(int64_t nloc, cudaStream_t st, const int* l2g, const double* g, double* loc) {
  ++g_launches;
  scatter_global<<<kRedBlocks * 2, 256, 0, st>>>(nloc, l2g, g, loc);
}

void launch_gather(int ndof, cudaStream_t st, const int64_t* owner, const double* loc, double* g) {
  if (ndof == 0) return;
  ++g_launches;
  gather_global<<<kRedBlocks * 2, 256, 0, st>>>(ndof, owner, loc, g);
}

void launch_axpby(int64_t n, cudaStream_t st, double a, const double* x, double b, double* y) {
  ++g_launches;
  axpby<<<kRedBlocks * 2, 256, 0, st>>>(n, a, x, b, y);
}

int red_blocks() { return kRedBlocks; }

}  // namespace dev
}  // namespace mgiga
