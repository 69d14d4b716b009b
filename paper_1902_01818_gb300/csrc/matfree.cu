// Matrix-free residual of the finest level (the patch part of r = f - A u, Sec. 2,
// Eq. linear:system:0): the stiffness action sum_q grad phi_i(q) . G(q) grad u(q) evaluated at the
// Gauss points (p + 1 per element and direction, as in the assembly) by sum factorisation, with the
// geometric factors G = w |det J| J^{-1} J^{-T} computed on the fly from the control points of the
// geometry map, so that no band coefficient is read.
//
// A CTA takes a tile of TE^d elements of one patch and the window of the (TE + p)^d B-splines that
// are nonzero on them:
//   u (window) -> values and xi_0-derivatives at the xi_0 points       (contract direction 0)
//             -> ... one direction at a time ... -> parameter gradient at every point
//   flux F = (w / |det J|) adj(J) (adj(J)^T grad u)                       (pointwise)
//   F -> back through the directions in reverse, with the transposed 1D tables
// and writes the window's partial sums (the contributions of its own elements) to a scratch buffer;
// a second kernel adds, for every position, the partials of the (at most 2^d when TE >= p) windows
// that contain it, in tile order.  Every sum is taken in a fixed order: the result does not depend on
// the launch or the scheduling.
//
// Assumptions checked on the host: maximal smoothness (element e of a direction carries the
// B-splines e .. e + p), and a geometry map that is one polynomial piece per patch (its knot vectors
// have no interior knots) of degree <= 2.  The within-patch SIPG terms, the cross-patch couplings and
// the conforming shared-DoF sums are applied afterwards by the same kernels as for the stored band.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "device.cuh"
#include "host.hpp"
#include "kernels.h"
#include "matfree.hpp"

namespace mgiga {
namespace dev {

namespace {

// elements per tile direction: 2D about 48-64 points per direction; 3D small enough that the
// per-column registers of the pointwise step fit (one thread per (x, y) point column)
template <int D, int P, typename T>
__host__ __device__ constexpr int mf_te() {
  if (D == 2) return P <= 1 ? 32 : P <= 3 ? 16 : P == 4 ? 12 : 8;
  if (sizeof(T) == 4) return P <= 1 ? 8 : P == 2 ? 6 : P <= 4 ? 4 : 3;
  return P <= 1 ? 6 : P == 2 ? 4 : P == 3 ? 3 : 2;
}

template <int D, int P, typename T>
__host__ __device__ constexpr int mf_threads() {
  constexpr int QX = mf_te<D, P, T>() * (P + 1);
  return D == 2 ? 256 : ((QX * QX + 31) / 32) * 32;
}

// shared memory (in T) of one CTA
template <int D, int P, int GM, typename T>
__host__ __device__ constexpr int mf_smem_elems() {
  constexpr int P1 = P + 1, TE = mf_te<D, P, T>(), NW = TE + P, QX = TE * P1;
  constexpr int TBL = QX * (2 * P1 + 1 + 2 * GM);
  constexpr int CP = D == 2 ? GM * GM * 2 : GM * GM * GM * 3;
  if (D == 2) return NW * NW + 2 * TBL + 2 * NW * QX + 2 * TE * P1 * QX + CP;
  return NW * NW * NW + 3 * TBL + 2 * NW * NW * QX + 3 * NW * QX * QX + CP;
}

template <typename T>
struct MfKArgs {
  const MfPatch* pp;
  int K;
  const T* B;        // per point x (p + 1): B-spline values
  const T* Dv;       //                      derivatives
  const T* w;        // per point: Gauss weight x element length
  const T* gB;       // per point x GM: geometry B-spline values (zero beyond its degree)
  const T* gD;       //                 derivatives
  const T* ctrl;     // geometry control points, per patch GM^d points of d values (zero padded)
  const unsigned char* dir;  // Dirichlet flag per local position
  const double* u;
  T* part;
  const Tile* tiles;
  const double* f;
  double* out;
};

// the window of u (Dirichlet entries and positions beyond the patch read as 0) and the 1D tables
// of the tile's elements (zero for elements beyond the patch: their points then carry no weight)
template <int D, int P, int GM, typename T>
__device__ __forceinline__ void mf_load(const MfKArgs<T>& a, const MfPatch& pp, const int* E, T* us, T* tb, T* cp) {
  constexpr int P1 = P + 1, TE = mf_te<D, P, T>(), NW = TE + P, QX = TE * P1;
  constexpr int TBL = QX * (2 * P1 + 1 + 2 * GM);
  const int tid = threadIdx.x, nthr = blockDim.x;
  constexpr int NWD = D == 2 ? NW * NW : NW * NW * NW;
  for (int i = tid; i < NWD; i += nthr) {
    const int j0 = i % NW, j1 = (i / NW) % NW, j2 = D == 3 ? i / (NW * NW) : 0;
    const int g0 = E[0] + j0, g1 = E[1] + j1, g2 = D == 3 ? E[2] + j2 : 0;
    T v = T(0);
    if (g0 < pp.N[0] && g1 < pp.N[1] && (D == 2 || g2 < pp.N[2])) {
      const int64_t pos = pp.off + g0 + (int64_t)pp.N[0] * (g1 + (int64_t)pp.N[1] * g2);
      if (!a.dir[pos]) v = (T)a.u[pos];
    }
    us[i] = v;
  }
  for (int dd = 0; dd < D; ++dd) {
    T* base = tb + dd * TBL;
    for (int i = tid; i < QX * P1; i += nthr) {
      const int qx = i / P1, l = i % P1;
      const int e = E[dd] + qx / P1;
      T b = T(0), dv = T(0);
      if (e < pp.ne[dd]) {
        const int64_t gq = pp.q0[dd] + (int64_t)e * P1 + qx % P1;
        b = a.B[gq * P1 + l];
        dv = a.Dv[gq * P1 + l];
      }
      base[i] = b;
      base[QX * P1 + i] = dv;
    }
    for (int qx = tid; qx < QX; qx += nthr) {
      const int e = E[dd] + qx / P1;
      const int64_t gq = pp.q0[dd] + (int64_t)e * P1 + qx % P1;
      const bool ok = e < pp.ne[dd];
      base[2 * QX * P1 + qx] = ok ? a.w[gq] : T(0);
      for (int g = 0; g < GM; ++g) {
        base[2 * QX * P1 + QX + qx * GM + g] = ok ? a.gB[gq * GM + g] : T(0);
        base[2 * QX * P1 + QX + QX * GM + qx * GM + g] = ok ? a.gD[gq * GM + g] : T(0);
      }
    }
  }
  constexpr int CP = D == 2 ? GM * GM * 2 : GM * GM * GM * 3;
  for (int i = tid; i < CP; i += nthr) cp[i] = a.ctrl[pp.ctrl + i];
}

// the CTA's patch and tile; E: first element of the tile per direction
template <int D, int TE>
__device__ __forceinline__ int mf_tile_of(const MfPatch* pp, int K, int* E, int* t_out) {
  int k = 0;
  while (k + 1 < K && (int)blockIdx.x >= pp[k + 1].tile0) ++k;
  const int t = (int)blockIdx.x - pp[k].tile0;
  E[0] = (t % pp[k].nt[0]) * TE;
  E[1] = ((t / pp[k].nt[0]) % pp[k].nt[1]) * TE;
  E[2] = D == 3 ? (t / (pp[k].nt[0] * pp[k].nt[1])) * TE : 0;
  *t_out = t;
  return k;
}

template <int P, int GM, typename T>
__global__ void __launch_bounds__(256) mf_tile_2d(MfKArgs<T> a) {
  constexpr int P1 = P + 1, TE = mf_te<2, P, T>(), NW = TE + P, QX = TE * P1;
  constexpr int TBL = QX * (2 * P1 + 1 + 2 * GM);
  extern __shared__ __align__(16) unsigned char mf_sm[];
  T* us = reinterpret_cast<T*>(mf_sm);  // [NW][NW]
  T* tb = us + NW * NW;                  // per direction: B [QX][P1], D [QX][P1], w [QX], gB [QX][GM], gD [QX][GM]
  T* VA = tb + 2 * TBL;                  // [NW][QX]: u contracted along xi_0 with the values
  T* VD = VA + NW * QX;                  //           ... with the derivatives
  T* WpD = VD + NW * QX;                 // [TE][P1][QX]: per element row, the back-contracted flux
  T* WpA = WpD + TE * P1 * QX;
  T* cp = WpA + TE * P1 * QX;            // control points [GM][GM][2]
  int E[3], t;
  const int k = mf_tile_of<2, TE>(a.pp, a.K, E, &t);
  const MfPatch pp = a.pp[k];
  mf_load<2, P, GM, T>(a, pp, E, us, tb, cp);
  __syncthreads();
  const T* B0 = tb;
  const T* D0 = tb + QX * P1;
  const T* w0 = tb + 2 * QX * P1;
  const T* gB0 = w0 + QX;
  const T* gD0 = gB0 + QX * GM;
  const T* B1 = tb + TBL;
  const T* D1 = B1 + QX * P1;
  const T* w1 = B1 + 2 * QX * P1;
  const T* gB1 = w1 + QX;
  const T* gD1 = gB1 + QX * GM;
  const int tid = threadIdx.x, nthr = blockDim.x;
  // direction 0: window rows j1 at the xi_0 points
  for (int i = tid; i < NW * QX; i += nthr) {
    const int j1 = i / QX, qx = i % QX, e = qx / P1;
    T sa = T(0), sd = T(0);
#pragma unroll
    for (int l = 0; l < P1; ++l) {
      const T uv = us[j1 * NW + e + l];
      sa += B0[qx * P1 + l] * uv;
      sd += D0[qx * P1 + l] * uv;
    }
    VA[i] = sa;
    VD[i] = sd;
  }
  __syncthreads();
  // direction 1, the flux at each point and its contraction back along xi_1, per (x point, element row)
  for (int i = tid; i < QX * TE; i += nthr) {
    const int qx = i % QX, ey = i / QX;
    T H0[GM][2], H1[GM][2];  // Jacobian columns along the xi_0 point: sums over the xi_0 control index
#pragma unroll
    for (int i1 = 0; i1 < GM; ++i1)
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int i0 = 0; i0 < GM; ++i0) {
          const T c = cp[(i0 + GM * i1) * 2 + x];
          s0 += c * gD0[qx * GM + i0];
          s1 += c * gB0[qx * GM + i0];
        }
        H0[i1][x] = s0;
        H1[i1][x] = s1;
      }
    T va[P1], vd[P1], wd[P1], wa[P1];
#pragma unroll
    for (int l = 0; l < P1; ++l) {
      va[l] = VA[(ey + l) * QX + qx];
      vd[l] = VD[(ey + l) * QX + qx];
      wd[l] = T(0);
      wa[l] = T(0);
    }
    const T wx = w0[qx];
#pragma unroll
    for (int j = 0; j < P1; ++j) {
      const int qy = ey * P1 + j;
      T gx = T(0), gy = T(0);
#pragma unroll
      for (int l = 0; l < P1; ++l) {
        gx += B1[qy * P1 + l] * vd[l];
        gy += D1[qy * P1 + l] * va[l];
      }
      T J00 = T(0), J10 = T(0), J01 = T(0), J11 = T(0);
#pragma unroll
      for (int i1 = 0; i1 < GM; ++i1) {
        const T b = gB1[qy * GM + i1], dv = gD1[qy * GM + i1];
        J00 += H0[i1][0] * b;
        J10 += H0[i1][1] * b;
        J01 += H1[i1][0] * dv;
        J11 += H1[i1][1] * dv;
      }
      const T det = J00 * J11 - J01 * J10;
      const T wq = wx * w1[qy];
      const T s = wq == T(0) ? T(0) : wq / fabs(det);
      // y = adj(J)^T g, F = s adj(J) y  (adj(J) = det J^{-1})
      const T y0 = J11 * gx - J10 * gy, y1 = J00 * gy - J01 * gx;
      const T Fx = s * (J11 * y0 - J01 * y1), Fy = s * (J00 * y1 - J10 * y0);
#pragma unroll
      for (int l = 0; l < P1; ++l) {
        wd[l] += B1[qy * P1 + l] * Fx;
        wa[l] += D1[qy * P1 + l] * Fy;
      }
    }
#pragma unroll
    for (int l = 0; l < P1; ++l) {
      WpD[(ey * P1 + l) * QX + qx] = wd[l];
      WpA[(ey * P1 + l) * QX + qx] = wa[l];
    }
  }
  __syncthreads();
  // per window row: the element rows' parts in ascending order
  for (int i = tid; i < NW * QX; i += nthr) {
    const int j1 = i / QX, qx = i % QX;
    T sd = T(0), sa = T(0);
    for (int ey = max(0, j1 - P); ey <= min(TE - 1, j1); ++ey) {
      sd += WpD[(ey * P1 + j1 - ey) * QX + qx];
      sa += WpA[(ey * P1 + j1 - ey) * QX + qx];
    }
    VD[i] = sd;
    VA[i] = sa;
  }
  __syncthreads();
  // direction 0 back: the window's partial sums
  T* dst = a.part + pp.pbase + (int64_t)t * (NW * NW);
  for (int i = tid; i < NW * NW; i += nthr) {
    const int j0 = i % NW, j1 = i / NW;
    T s = T(0);
    for (int ex = max(0, j0 - P); ex <= min(TE - 1, j0); ++ex) {
      const int l = j0 - ex;
#pragma unroll
      for (int j = 0; j < P1; ++j) {
        const int qx = ex * P1 + j;
        s += D0[qx * P1 + l] * VD[j1 * QX + qx] + B0[qx * P1 + l] * VA[j1 * QX + qx];
      }
    }
    dst[i] = s;
  }
}

template <int P, int GM, typename T>
__global__ void __launch_bounds__(mf_threads<3, P, T>()) mf_tile_3d(MfKArgs<T> a) {
  constexpr int P1 = P + 1, TE = mf_te<3, P, T>(), NW = TE + P, QX = TE * P1;
  constexpr int TBL = QX * (2 * P1 + 1 + 2 * GM);
  extern __shared__ __align__(16) unsigned char mf_sm[];
  T* us = reinterpret_cast<T*>(mf_sm);  // [NW][NW][NW]
  T* tb = us + NW * NW * NW;             // per direction: B, D, w, gB, gD as in 2D
  T* VA = tb + 3 * TBL;                  // [NW][NW][QX] (j2, j1, x point)
  T* VD = VA + NW * NW * QX;
  T* AX = VD + NW * NW * QX;             // [NW][QX][QX] (j2, y point, x point): for d/dxi_0
  T* AY = AX + NW * QX * QX;             //                                      for d/dxi_1
  T* AZ = AY + NW * QX * QX;             //                                      for d/dxi_2
  T* cp = AZ + NW * QX * QX;             // control points [GM][GM][GM][3]
  int E[3], t;
  const int k = mf_tile_of<3, TE>(a.pp, a.K, E, &t);
  const MfPatch pp = a.pp[k];
  mf_load<3, P, GM, T>(a, pp, E, us, tb, cp);
  __syncthreads();
  const T* Bt[3];
  const T* Dt[3];
  const T* wt[3];
  const T* gBt[3];
  const T* gDt[3];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    Bt[dd] = tb + dd * TBL;
    Dt[dd] = Bt[dd] + QX * P1;
    wt[dd] = Bt[dd] + 2 * QX * P1;
    gBt[dd] = wt[dd] + QX;
    gDt[dd] = gBt[dd] + QX * GM;
  }
  const int tid = threadIdx.x, nthr = blockDim.x;
  // direction 0
  for (int i = tid; i < NW * NW * QX; i += nthr) {
    const int qx = i % QX, j12 = i / QX, e = qx / P1;
    T sa = T(0), sd = T(0);
#pragma unroll
    for (int l = 0; l < P1; ++l) {
      const T uv = us[j12 * NW + e + l];
      sa += Bt[0][qx * P1 + l] * uv;
      sd += Dt[0][qx * P1 + l] * uv;
    }
    VA[i] = sa;
    VD[i] = sd;
  }
  __syncthreads();
  // direction 1
  for (int i = tid; i < NW * QX * QX; i += nthr) {
    const int qx = i % QX, qy = (i / QX) % QX, j2 = i / (QX * QX), e = qy / P1;
    T sx = T(0), sy = T(0), sz = T(0);
#pragma unroll
    for (int l = 0; l < P1; ++l) {
      const int src = ((j2 * NW) + e + l) * QX + qx;
      const T b = Bt[1][qy * P1 + l], dv = Dt[1][qy * P1 + l];
      sx += b * VD[src];
      sy += dv * VA[src];
      sz += b * VA[src];
    }
    AX[i] = sx;
    AY[i] = sy;
    AZ[i] = sz;
  }
  __syncthreads();
  // direction 2, the flux, and back along xi_2: one thread per (x, y) point column; the column is
  // read and then overwritten by its own thread only
  if (tid < QX * QX) {
    const int qx = tid % QX, qy = tid / QX;
    T H0[GM][3], H1[GM][3], H2[GM][3];  // Jacobian columns along the (x, y) column: sums over i0, i1
#pragma unroll
    for (int i2 = 0; i2 < GM; ++i2)
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
        for (int i1 = 0; i1 < GM; ++i1)
#pragma unroll
          for (int i0 = 0; i0 < GM; ++i0) {
            const T c = cp[(i0 + GM * (i1 + GM * i2)) * 3 + x];
            const T b0 = gBt[0][qx * GM + i0], d0 = gDt[0][qx * GM + i0];
            const T b1 = gBt[1][qy * GM + i1], d1 = gDt[1][qy * GM + i1];
            s0 += c * (d0 * b1);
            s1 += c * (b0 * d1);
            s2 += c * (b0 * b1);
          }
        H0[i2][x] = s0;
        H1[i2][x] = s1;
        H2[i2][x] = s2;
      }
    T ax[NW], ay[NW], az[NW], rx[NW], ry[NW], rz[NW];
#pragma unroll
    for (int j2 = 0; j2 < NW; ++j2) {
      const int c = (j2 * QX + qy) * QX + qx;
      ax[j2] = AX[c];
      ay[j2] = AY[c];
      az[j2] = AZ[c];
      rx[j2] = T(0);
      ry[j2] = T(0);
      rz[j2] = T(0);
    }
    const T wxy = wt[0][qx] * wt[1][qy];
#pragma unroll
    for (int ez = 0; ez < TE; ++ez)
#pragma unroll
      for (int j = 0; j < P1; ++j) {
        const int qz = ez * P1 + j;
        T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
        for (int l = 0; l < P1; ++l) {
          const T b = Bt[2][qz * P1 + l], dv = Dt[2][qz * P1 + l];
          gx += b * ax[ez + l];
          gy += b * ay[ez + l];
          gz += dv * az[ez + l];
        }
        T J[3][3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
          for (int i2 = 0; i2 < GM; ++i2) {
            const T b = gBt[2][qz * GM + i2], dv = gDt[2][qz * GM + i2];
            s0 += H0[i2][x] * b;
            s1 += H1[i2][x] * b;
            s2 += H2[i2][x] * dv;
          }
          J[x][0] = s0;
          J[x][1] = s1;
          J[x][2] = s2;
        }
        // adjugate M = det J^{-1}
        const T M00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const T M01 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        const T M02 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        const T M10 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const T M11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        const T M12 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        const T M20 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const T M21 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        const T M22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const T det = J[0][0] * M00 + J[0][1] * M10 + J[0][2] * M20;
        const T wq = wxy * wt[2][qz];
        const T s = wq == T(0) ? T(0) : wq / fabs(det);
        const T y0 = M00 * gx + M10 * gy + M20 * gz;
        const T y1 = M01 * gx + M11 * gy + M21 * gz;
        const T y2 = M02 * gx + M12 * gy + M22 * gz;
        const T Fx = s * (M00 * y0 + M01 * y1 + M02 * y2);
        const T Fy = s * (M10 * y0 + M11 * y1 + M12 * y2);
        const T Fz = s * (M20 * y0 + M21 * y1 + M22 * y2);
#pragma unroll
        for (int l = 0; l < P1; ++l) {
          const T b = Bt[2][qz * P1 + l], dv = Dt[2][qz * P1 + l];
          rx[ez + l] += b * Fx;
          ry[ez + l] += b * Fy;
          rz[ez + l] += dv * Fz;
        }
      }
#pragma unroll
    for (int j2 = 0; j2 < NW; ++j2) {
      const int c = (j2 * QX + qy) * QX + qx;
      AX[c] = rx[j2];
      AY[c] = ry[j2];
      AZ[c] = rz[j2];
    }
  }
  __syncthreads();
  // direction 1 back: (j2, j1, x point), the element rows covering j1 in ascending order
  for (int i = tid; i < NW * NW * QX; i += nthr) {
    const int qx = i % QX, j1 = (i / QX) % NW, j2 = i / (QX * NW);
    T sd = T(0), sa = T(0);
    for (int ey = max(0, j1 - P); ey <= min(TE - 1, j1); ++ey) {
      const int l = j1 - ey;
#pragma unroll
      for (int j = 0; j < P1; ++j) {
        const int qy = ey * P1 + j;
        const int c = (j2 * QX + qy) * QX + qx;
        const T b = Bt[1][qy * P1 + l], dv = Dt[1][qy * P1 + l];
        sd += b * AX[c];
        sa += dv * AY[c] + b * AZ[c];
      }
    }
    VD[i] = sd;
    VA[i] = sa;
  }
  __syncthreads();
  // direction 0 back: the window's partial sums
  T* dst = a.part + pp.pbase + (int64_t)t * (NW * NW * NW);
  for (int i = tid; i < NW * NW * NW; i += nthr) {
    const int j0 = i % NW, j12 = i / NW;
    T s = T(0);
    for (int ex = max(0, j0 - P); ex <= min(TE - 1, j0); ++ex) {
      const int l = j0 - ex;
#pragma unroll
      for (int j = 0; j < P1; ++j) {
        const int qx = ex * P1 + j;
        s += Dt[0][qx * P1 + l] * VD[j12 * QX + qx] + Bt[0][qx * P1 + l] * VA[j12 * QX + qx];
      }
    }
    dst[i] = s;
  }
}

// out = f - (sum of the window partials containing the position), Dirichlet rows: out = f (their
// band rows are zero); one thread per position of a 256-position tile
template <int D, int P, typename T>
__global__ void __launch_bounds__(kTile) mf_gather(MfKArgs<T> a) {
  constexpr int TE = mf_te<D, P, T>(), NW = TE + P;
  const Tile tl = a.tiles[blockIdx.x];
  const int i = threadIdx.x;
  if (i >= tl.count) return;
  const int64_t pos = tl.start + i;
  if (a.dir[pos]) {
    a.out[pos] = a.f[pos];
    return;
  }
  const MfPatch pp = a.pp[tl.patch];
  int64_t rem = pos - pp.off;
  int ix[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  ix[0] = (int)(rem % pp.N[0]);
  rem /= pp.N[0];
  ix[1] = (int)(rem % pp.N[1]);
  ix[2] = D == 3 ? (int)(rem / pp.N[1]) : 0;
#pragma unroll
  for (int dd = 0; dd < D; ++dd) {
    const int first = ix[dd] - NW + 1;
    lo[dd] = first <= 0 ? 0 : (first + TE - 1) / TE;
    hi[dd] = min(pp.nt[dd] - 1, ix[dd] / TE);
  }
  T s = T(0);
  for (int t2 = lo[2]; t2 <= hi[2]; ++t2)
    for (int t1 = lo[1]; t1 <= hi[1]; ++t1)
      for (int t0 = lo[0]; t0 <= hi[0]; ++t0) {
        const int64_t tile = t0 + (int64_t)pp.nt[0] * (t1 + (int64_t)pp.nt[1] * t2);
        const int w = (ix[0] - t0 * TE) + NW * ((ix[1] - t1 * TE) + NW * (D == 3 ? ix[2] - t2 * TE : 0));
        s += a.part[pp.pbase + tile * (D == 2 ? NW * NW : NW * NW * NW) + w];
      }
  a.out[pos] = a.f[pos] - (double)s;
}

template <int D, int P, int GM, typename T>
void mf_launch_t(const MfDev& m, cudaStream_t st, const double* u, const double* f, double* out, int ntiles,
                 const Tile* tiles) {
  MfKArgs<T> a;
  a.pp = m.pp;
  a.K = m.K;
  a.B = static_cast<const T*>(m.B);
  a.Dv = static_cast<const T*>(m.Dv);
  a.w = static_cast<const T*>(m.w);
  a.gB = static_cast<const T*>(m.gB);
  a.gD = static_cast<const T*>(m.gD);
  a.ctrl = static_cast<const T*>(m.ctrl);
  a.dir = m.dir;
  a.u = u;
  a.part = static_cast<T*>(m.part);
  a.tiles = tiles;
  a.f = f;
  a.out = out;
  constexpr int smem = mf_smem_elems<D, P, GM, T>() * (int)sizeof(T);
  static bool attr = false;  // per process: the attribute belongs to the kernel, any device
  if (D == 2) {
    if (!attr) {
      cudaFuncSetAttribute(mf_tile_2d<P, GM, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr = true;
    }
    count_launch();
    mf_tile_2d<P, GM, T><<<m.ntile, 256, smem, st>>>(a);
  } else {
    if (!attr) {
      cudaFuncSetAttribute(mf_tile_3d<P, GM, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr = true;
    }
    count_launch();
    mf_tile_3d<P, GM, T><<<m.ntile, mf_threads<3, P, T>(), smem, st>>>(a);
  }
  count_launch();
  mf_gather<D, P, T><<<ntiles, kTile, 0, st>>>(a);
}

template <int D, int P, typename T>
void mf_launch_g(const MfDev& m, cudaStream_t st, const double* u, const double* f, double* out, int ntiles,
                 const Tile* tiles) {
  if (m.GM == 2) mf_launch_t<D, P, 2, T>(m, st, u, f, out, ntiles, tiles);
  else mf_launch_t<D, P, 3, T>(m, st, u, f, out, ntiles, tiles);
}

template <int D, typename T>
void mf_launch_p(int p, const MfDev& m, cudaStream_t st, const double* u, const double* f, double* out, int ntiles,
                 const Tile* tiles) {
  switch (p) {
    case 1: mf_launch_g<D, 1, T>(m, st, u, f, out, ntiles, tiles); break;
    case 2: mf_launch_g<D, 2, T>(m, st, u, f, out, ntiles, tiles); break;
    case 3: mf_launch_g<D, 3, T>(m, st, u, f, out, ntiles, tiles); break;
    case 4: mf_launch_g<D, 4, T>(m, st, u, f, out, ntiles, tiles); break;
    case 5: mf_launch_g<D, 5, T>(m, st, u, f, out, ntiles, tiles); break;
    default: mf_launch_g<D, 6, T>(m, st, u, f, out, ntiles, tiles); break;
  }
}

template <int D, int P, typename T>
void mf_geometry(int* te, int* nthreads) {
  *te = mf_te<D, P, T>();
  *nthreads = D == 2 ? 256 : mf_threads<D, P, T>();
}

}  // namespace

int mf_tile_elems(int d, int p, bool f32) {
  int te = 0, nt = 0;
#define MF_CASE(D, P)                                              \
  if (d == D && p == P) {                                          \
    if (f32) mf_geometry<D, P, float>(&te, &nt);                   \
    else mf_geometry<D, P, double>(&te, &nt);                      \
  }
  MF_CASE(2, 1) MF_CASE(2, 2) MF_CASE(2, 3) MF_CASE(2, 4) MF_CASE(2, 5) MF_CASE(2, 6)
  MF_CASE(3, 1) MF_CASE(3, 2) MF_CASE(3, 3) MF_CASE(3, 4) MF_CASE(3, 5) MF_CASE(3, 6)
#undef MF_CASE
  return te;
}

bool mf_supported(const Problem& pr, std::string* why) {
  if (pr.p < 1 || pr.p > 6 || (pr.d != 2 && pr.d != 3)) {
    if (why) *why = "degree 1..6 in 2D or 3D";
    return false;
  }
  for (int k = 0; k < pr.K; ++k) {
    if (pr.deg(k) != pr.p) {
      if (why) *why = "one degree for all patches";
      return false;
    }
    const Geometry& g = pr.geo[k];
    if (g.q > 2) {
      if (why) *why = "geometry degree <= 2 (patch " + std::to_string(k) + ")";
      return false;
    }
    for (int a = 0; a < pr.d; ++a)
      if (breakpoints(g.knots[a]).size() != 2) {
        if (why) *why = "a geometry map that is one polynomial piece per patch (patch " + std::to_string(k) + ")";
        return false;
      }
  }
  return true;
}

MfHost mf_build_host(const Problem& pr, const Level& F, bool f32) {
  MfHost h;
  const int d = pr.d, p = pr.p, P1 = p + 1;
  int GM = 2;
  for (int k = 0; k < pr.K; ++k) GM = std::max(GM, pr.geo[k].q + 1);
  h.GM = GM;
  h.te = mf_tile_elems(d, p, f32);
  const int TE = h.te, NW = TE + p;
  const int64_t win = d == 2 ? (int64_t)NW * NW : (int64_t)NW * NW * NW;
  double xg[16], wg[16];
  gauss_legendre(P1, xg, wg);
  int64_t nq = 0, pbase = 0;
  int tile0 = 0;
  for (int k = 0; k < F.K; ++k) {
    MfPatch m{};
    m.off = F.off[k];
    const Geometry& g = pr.geo[k];
    for (int a = 0; a < 3; ++a) {
      m.N[a] = F.N[k][a];
      m.ne[a] = 1;
      m.nt[a] = 1;
      m.q0[a] = nq;
      if (a >= d) continue;
      const Vec& t = F.knots[k][a];
      const Vec z = breakpoints(t);
      m.ne[a] = (int)z.size() - 1;
      m.nt[a] = (m.ne[a] + TE - 1) / TE;
      if (m.N[a] != m.ne[a] + p) throw SetupError(1, "matrix-free residual: knot vectors of maximal smoothness needed");
      double N[16], dN[16];
      for (int e = 0; e < m.ne[a]; ++e) {
        const double lo = z[e], hl = z[e + 1] - z[e];
        const int s = find_span(t, p, lo + 0.5 * hl);
        if (s - p != e) throw SetupError(1, "matrix-free residual: knot vectors of maximal smoothness needed");
        for (int j = 0; j < P1; ++j) {
          const double x = lo + hl * xg[j];
          h.w.push_back(hl * wg[j]);
          basis_on_span(t, p, s, x, N, dN);
          for (int l = 0; l < P1; ++l) {
            h.B.push_back(N[l]);
            h.Dv.push_back(dN[l]);
          }
          const int gs = find_span(g.knots[a], g.q, x);
          basis_on_span(g.knots[a], g.q, gs, x, N, dN);
          for (int l = 0; l < GM; ++l) {
            h.gB.push_back(l <= g.q ? N[l] : 0.0);
            h.gD.push_back(l <= g.q ? dN[l] : 0.0);
          }
          ++nq;
        }
      }
    }
    // control points of the single geometry piece, padded to GM per direction
    m.ctrl = (int64_t)h.ctrl.size();
    const int n2 = d == 3 ? GM : 1;
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i1 = 0; i1 < GM; ++i1)
        for (int i0 = 0; i0 < GM; ++i0)
          for (int x = 0; x < d; ++x) {
            const bool ok = i0 <= g.q && i1 <= g.q && i2 <= (d == 3 ? g.q : 0);
            h.ctrl.push_back(ok ? g.ctrl[(i0 + (size_t)g.ncp[0] * (i1 + (size_t)g.ncp[1] * i2)) * d + x] : 0.0);
          }
    int64_t ntile = 1;
    for (int a = 0; a < d; ++a) ntile *= m.nt[a];
    m.tile0 = tile0;
    m.pbase = pbase;
    tile0 += (int)ntile;
    pbase += ntile * win;
    h.pp.push_back(m);
  }
  h.ntile = tile0;
  h.part_n = pbase;
  const int64_t ntot = tile0;
  // kernel work per launch: FMAs of the sum-factorised passes and of the pointwise step (2 flops each)
  const int QX = TE * P1;
  double fma_tile;
  if (d == 2) {
    fma_tile = (double)NW * QX * 2 * P1 + (double)QX * TE * P1 * (4.0 * P1 + 12.0) +
               (double)NW * NW * P1 * P1 * 2;
  } else {
    fma_tile = (double)NW * NW * QX * 2 * P1 + (double)NW * QX * QX * 3 * P1 +
               (double)QX * QX * TE * P1 * (6.0 * P1 + 9.0 * GM + 45.0) + (double)NW * NW * QX * P1 * P1 * 3 +
               (double)NW * NW * NW * P1 * P1 * 2;
  }
  h.flops = 2.0 * fma_tile * (double)ntot;
  return h;
}

void mf_launch(int d, int p, bool f32, const MfDev& m, cudaStream_t st, const double* u, const double* f, double* out,
               int ntiles, const Tile* tiles) {
  if (d == 2) {
    if (f32) mf_launch_p<2, float>(p, m, st, u, f, out, ntiles, tiles);
    else mf_launch_p<2, double>(p, m, st, u, f, out, ntiles, tiles);
  } else {
    if (f32) mf_launch_p<3, float>(p, m, st, u, f, out, ntiles, tiles);
    else mf_launch_p<3, double>(p, m, st, u, f, out, ntiles, tiles);
  }
}

}  // namespace dev
}  // namespace mgiga
