// Set-up of the level operators on the GPU (Sec. 2, 3):
//   * the patch stiffness of the finest level, K_ij = sum_q w_q |det J| (J^{-T} grad^ B_i).(J^{-T} grad^ B_j)
//     (Sec. 2, Eq. linear:system:0), p + 1 Gauss points per element and direction, one CTA per
//     element, sum-factorised over the directions, added into the offset-major band;
//   * the SIPG interface terms that couple functions of one patch (Sec. 3, Eq. model:discr2), computed
//     on the host with the cross-patch blocks and added here;
//   * the strong Dirichlet condition (rows and columns of Dirichlet functions zeroed);
//   * the Galerkin coarse operators A_{l-1} = P^T A_l P (Sec. 3, Eq. a:galerkin) of the patch bands,
//     one direction at a time.
// Every band entry is the sum of its contributions in a fixed order: the elements are coloured by
// their indices modulo p + 1 in every direction, so that the elements of one launch touch disjoint
// rows, and the colours are launched one after another.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "device.cuh"
#include "host.hpp"
#include "kernels.h"
#include "setup_gpu.hpp"

namespace mgiga {
namespace dev {

namespace {

#define SCK(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) throw std::runtime_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// quadrature data of one direction of one patch: elements [e0, e0 + ne) of the span table,
// quadrature points [q0, q0 + ne nq) of the point tables
struct QTab {
  int64_t e0, q0;
  int ne, pad;
};

struct PatchGeo {
  int64_t ctrl;  // offset (in doubles) of the first control point (dim doubles each)
  int ncp[3];
  int q;         // degree of the geometry splines
};

struct AsmArgs {
  const QTab* qt;          // [K * 3]
  const int* span;         // per element: knot span (solution knots)
  const double* w;         // per quadrature point: weight x element length
  const double* B;         // per point x (p + 1): B-spline values
  const double* D;         //                      derivatives
  const int* gspan;        // per point: geometry knot span
  const double* gB;        // per point x G1: geometry B-spline values
  const double* gD;        //                   derivatives
  int G1;                  // stride of gB / gD (largest geometry degree + 1)
  const PatchGeo* geo;
  const double* ctrl;
  const PatchMeta* pm;
  const int* cta_ptr;      // CTA prefix over the patches for the launched colour (K + 1)
  double* bt;              // the band accumulated row-major, bt[row * nb + o] (an element's entries of
                           // one row share cache lines), transposed into the offset-major band at the end
  int64_t nloc;
  int c0, c1, c2;          // the colour: element index residues modulo p + 1
};

// Jacobian J[a d + b] = dX_a / dxi_b of the geometry at the point with per-direction point indices
template <int DIM>
__device__ __forceinline__ void geo_jacobian(const AsmArgs& a, int k, const int64_t* qi, double* J) {
  const PatchGeo g = a.geo[k];
  for (int i = 0; i < DIM * DIM; ++i) J[i] = 0.0;
  int gs[3];
  for (int dd = 0; dd < DIM; ++dd) gs[dd] = a.gspan[qi[dd]];
  const int n2 = DIM == 3 ? g.q + 1 : 1;
  for (int i2 = 0; i2 < n2; ++i2)
    for (int i1 = 0; i1 <= g.q; ++i1)
      for (int i0 = 0; i0 <= g.q; ++i0) {
        const int I0 = gs[0] - g.q + i0, I1 = gs[1] - g.q + i1, I2 = DIM == 3 ? gs[2] - g.q + i2 : 0;
        const double* c = a.ctrl + g.ctrl + (I0 + (int64_t)g.ncp[0] * (I1 + (int64_t)g.ncp[1] * I2)) * DIM;
        const double b0 = a.gB[qi[0] * a.G1 + i0], d0 = a.gD[qi[0] * a.G1 + i0];
        const double b1 = a.gB[qi[1] * a.G1 + i1], d1 = a.gD[qi[1] * a.G1 + i1];
        const double b2 = DIM == 3 ? a.gB[qi[2] * a.G1 + i2] : 1.0, d2 = DIM == 3 ? a.gD[qi[2] * a.G1 + i2] : 0.0;
        const double der[3] = {d0 * b1 * b2, b0 * d1 * b2, b0 * b1 * d2};
        for (int x = 0; x < DIM; ++x)
          for (int y = 0; y < DIM; ++y) J[x * DIM + y] += der[y] * c[x];
      }
}

// geometric factors C_ab = w |det J| (J^{-1} J^{-T})_ab, all DIM^2 of them
template <int DIM>
__device__ __forceinline__ void geo_factors(const double* J, double w, double* C) {
  double Ji[9];
  double det;
  if (DIM == 2) {
    det = J[0] * J[3] - J[1] * J[2];
    Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
  } else {
    const double c00 = J[4] * J[8] - J[5] * J[7];
    const double c01 = J[5] * J[6] - J[3] * J[8];
    const double c02 = J[3] * J[7] - J[4] * J[6];
    det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    Ji[0] = c00 / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det; Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    Ji[3] = c01 / det; Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[6] = c02 / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det; Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  }
  const double s = w * fabs(det);
  for (int x = 0; x < DIM; ++x)
    for (int y = 0; y < DIM; ++y) {
      double v = 0.0;
      for (int c = 0; c < DIM; ++c) v += Ji[x * DIM + c] * Ji[y * DIM + c];
      C[x * DIM + y] = s * v;
    }
}

// CTA -> (patch, element) of the launched colour
template <int P1>
__device__ __forceinline__ int element_of(const AsmArgs& a, int dim, int* e) {
  int b = blockIdx.x, k = 0;
  while (b >= a.cta_ptr[k + 1]) ++k;
  int loc = b - a.cta_ptr[k];
  const int c[3] = {a.c0, a.c1, a.c2};
  for (int dd = 0; dd < dim; ++dd) {
    const int n = (a.qt[k * 3 + dd].ne - c[dd] + P1 - 1) / P1;
    e[dd] = c[dd] + P1 * (loc % n);
    loc /= n;
  }
  return k;
}

template <int P>
__global__ void __launch_bounds__(128) stiffness_2d(AsmArgs a) {
  constexpr int P1 = P + 1, NQ = P + 1, L2 = P1 * P1, W = 2 * P + 1;
  __shared__ double sC[NQ * NQ][4];
  __shared__ double sV[2][NQ][P1], sD[2][NQ][P1];
  __shared__ double sU[4][NQ][L2];
  int e[3];
  const int k = element_of<P1>(a, 2, e);
  const QTab t0 = a.qt[k * 3], t1 = a.qt[k * 3 + 1];
  const int tid = threadIdx.x;
  for (int i = tid; i < NQ * P1; i += blockDim.x) {
    const int q = i / P1, l = i % P1;
    const int64_t i0 = (t0.q0 + (int64_t)e[0] * NQ + q) * P1 + l, i1 = (t1.q0 + (int64_t)e[1] * NQ + q) * P1 + l;
    sV[0][q][l] = a.B[i0]; sD[0][q][l] = a.D[i0];
    sV[1][q][l] = a.B[i1]; sD[1][q][l] = a.D[i1];
  }
  for (int qq = tid; qq < NQ * NQ; qq += blockDim.x) {
    const int q0 = qq % NQ, q1 = qq / NQ;
    const int64_t qi[3] = {t0.q0 + (int64_t)e[0] * NQ + q0, t1.q0 + (int64_t)e[1] * NQ + q1, 0};
    double J[4], C[4];
    geo_jacobian<2>(a, k, qi, J);
    geo_factors<2>(J, a.w[qi[0]] * a.w[qi[1]], C);
    for (int x = 0; x < 4; ++x) sC[qq][x] = C[x];
  }
  __syncthreads();
  // U_ab(q0, l1, m1) = sum_q1 C_ab(q0, q1) X1_a(q1, l1) X1_b(q1, m1); X_a is the derivative along
  // direction a, so its factor along xi_1 is the derivative for a = 1, the value for a = 0
  for (int i = tid; i < 4 * NQ * L2; i += blockDim.x) {
    const int ab = i / (NQ * L2), rem = i % (NQ * L2), q0 = rem / L2, lm = rem % L2;
    const int aa = ab >> 1, bb = ab & 1, l1 = lm / P1, m1 = lm % P1;
    double s = 0.0;
#pragma unroll
    for (int q1 = 0; q1 < NQ; ++q1) {
      const double xa = aa ? sD[1][q1][l1] : sV[1][q1][l1];
      const double xb = bb ? sD[1][q1][m1] : sV[1][q1][m1];
      s += sC[q0 + NQ * q1][ab] * xa * xb;
    }
    sU[ab][q0][lm] = s;
  }
  __syncthreads();
  // K_e(l, m) = sum_q0 sum_ab X0_a(q0, l0) X0_b(q0, m0) U_ab(q0, l1, m1), added to the band row of l
  const PatchMeta pm = a.pm[k];
  const int s0 = a.span[t0.e0 + e[0]] - P, s1 = a.span[t1.e0 + e[1]] - P;
  for (int i = tid; i < L2 * L2; i += blockDim.x) {
    const int l = i / L2, m = i % L2;
    const int l0 = l % P1, l1 = l / P1, m0 = m % P1, m1 = m / P1;
    const int lm = l1 * P1 + m1;
    double s = 0.0;
#pragma unroll
    for (int q0 = 0; q0 < NQ; ++q0) {
      const double a0 = sD[0][q0][l0], a1 = sV[0][q0][l0], b0 = sD[0][q0][m0], b1 = sV[0][q0][m0];
      s += a0 * (b0 * sU[0][q0][lm] + b1 * sU[1][q0][lm]) + a1 * (b0 * sU[2][q0][lm] + b1 * sU[3][q0][lm]);
    }
    const int64_t row = pm.off + (s0 + l0) + (int64_t)pm.N[0] * (s1 + l1);
    const int o = (m0 - l0 + P) + W * (m1 - l1 + P);
    a.bt[row * (W * W) + o] += s;
  }
}

// 3D: contract the q2 points first (T2), then, per pair of (xi_1, xi_2) row / column indices
// (L12, M12) with L12 <= M12 (C is symmetric), the q1 points into a 2 x 2 form along xi_0 (only
// "a = 0 or not" matters there) and the q0 points into the (p + 1)^2 block of K_e; the block of
// (M12, L12) is its transpose
template <int P>
__global__ void __launch_bounds__(256) stiffness_3d(AsmArgs a) {
  constexpr int P1 = P + 1, NQ = P + 1, L2 = P1 * P1, W = 2 * P + 1;
  extern __shared__ __align__(16) double s3[];
  double* sC = s3;                       // [NQ^3][9]
  double* sV = sC + NQ * NQ * NQ * 9;    // [3][NQ][P1]
  double* sD = sV + 3 * NQ * P1;         // [3][NQ][P1]
  double* sT = sD + 3 * NQ * P1;         // [9][NQ][NQ][L2]: q0, q1, (l2, m2)
  int e[3];
  const int k = element_of<P1>(a, 3, e);
  QTab t[3];
  for (int dd = 0; dd < 3; ++dd) t[dd] = a.qt[k * 3 + dd];
  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * NQ * P1; i += blockDim.x) {
    const int dd = i / (NQ * P1), q = (i / P1) % NQ, l = i % P1;
    const int64_t x = (t[dd].q0 + (int64_t)e[dd] * NQ + q) * P1 + l;
    sV[i] = a.B[x];
    sD[i] = a.D[x];
  }
  for (int qq = tid; qq < NQ * NQ * NQ; qq += blockDim.x) {
    const int q0 = qq % NQ, q1 = (qq / NQ) % NQ, q2 = qq / (NQ * NQ);
    const int64_t qi[3] = {t[0].q0 + (int64_t)e[0] * NQ + q0, t[1].q0 + (int64_t)e[1] * NQ + q1,
                           t[2].q0 + (int64_t)e[2] * NQ + q2};
    double J[9];
    geo_jacobian<3>(a, k, qi, J);
    geo_factors<3>(J, a.w[qi[0]] * a.w[qi[1]] * a.w[qi[2]], sC + (size_t)qq * 9);
  }
  __syncthreads();
  auto V = [&](int dd, int q, int l) { return sV[(dd * NQ + q) * P1 + l]; };
  auto Dv = [&](int dd, int q, int l) { return sD[(dd * NQ + q) * P1 + l]; };
  // T2_ab(q0, q1, l2, m2) = sum_q2 C_ab X2_a(q2, l2) X2_b(q2, m2)
  for (int i = tid; i < 9 * NQ * NQ * L2; i += blockDim.x) {
    const int ab = i / (NQ * NQ * L2), rem = i % (NQ * NQ * L2);
    const int q01 = rem / L2, lm = rem % L2, l2 = lm / P1, m2 = lm % P1;
    const int aa = ab / 3, bb = ab % 3;
    double s = 0.0;
#pragma unroll
    for (int q2 = 0; q2 < NQ; ++q2) {
      const double xa = aa == 2 ? Dv(2, q2, l2) : V(2, q2, l2);
      const double xb = bb == 2 ? Dv(2, q2, m2) : V(2, q2, m2);
      s += sC[(size_t)(q01 + NQ * NQ * q2) * 9 + ab] * xa * xb;
    }
    sT[(size_t)ab * NQ * NQ * L2 + rem] = s;
  }
  __syncthreads();
  const PatchMeta pm = a.pm[k];
  const int s0 = a.span[t[0].e0 + e[0]] - P, s1 = a.span[t[1].e0 + e[1]] - P, s2 = a.span[t[2].e0 + e[2]] - P;
  const int npair = L2 * (L2 + 1) / 2;
  for (int pi = tid; pi < npair; pi += blockDim.x) {
    // pair index -> (L12, M12), L12 <= M12
    int L12 = 0, rem = pi;
    while (rem >= L2 - L12) { rem -= L2 - L12; ++L12; }
    const int M12 = L12 + rem;
    const int l1 = L12 % P1, l2 = L12 / P1, m1 = M12 % P1, m2 = M12 / P1;
    double blk[P1][P1];
#pragma unroll
    for (int x = 0; x < P1; ++x)
#pragma unroll
      for (int y = 0; y < P1; ++y) blk[x][y] = 0.0;
    for (int q0 = 0; q0 < NQ; ++q0) {
      double v[9];
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) {
        const int aa = ab / 3, bb = ab % 3;
        double s = 0.0;
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1) {
          const double xa = aa == 1 ? Dv(1, q1, l1) : V(1, q1, l1);
          const double xb = bb == 1 ? Dv(1, q1, m1) : V(1, q1, m1);
          s += sT[(size_t)ab * NQ * NQ * L2 + (q0 + NQ * q1) * L2 + l2 * P1 + m2] * xa * xb;
        }
        v[ab] = s;
      }
      const double w00 = v[0], w01 = v[1] + v[2], w10 = v[3] + v[6], w11 = (v[4] + v[5]) + (v[7] + v[8]);
#pragma unroll
      for (int l0 = 0; l0 < P1; ++l0) {
        const double a0 = Dv(0, q0, l0), a1 = V(0, q0, l0);
#pragma unroll
        for (int m0 = 0; m0 < P1; ++m0) {
          const double b0 = Dv(0, q0, m0), b1 = V(0, q0, m0);
          blk[l0][m0] += a0 * (w00 * b0 + w01 * b1) + a1 * (w10 * b0 + w11 * b1);
        }
      }
    }
    const int64_t N0 = pm.N[0], N01 = (int64_t)pm.N[0] * pm.N[1];
#pragma unroll
    for (int l0 = 0; l0 < P1; ++l0)
#pragma unroll
      for (int m0 = 0; m0 < P1; ++m0) {
        if (L12 == M12 && m0 < l0) continue;  // a diagonal block: its upper half (and the mirror)
        const double val = blk[l0][m0];
        {  // (l, m)
          const int64_t row = pm.off + (s0 + l0) + N0 * (s1 + l1) + N01 * (s2 + l2);
          const int o = (m0 - l0 + P) + W * (m1 - l1 + P) + W * W * (m2 - l2 + P);
          a.bt[row * (W * W * W) + o] += val;
        }
        if (L12 != M12 || m0 != l0) {  // (m, l)
          const int64_t row = pm.off + (s0 + m0) + N0 * (s1 + m1) + N01 * (s2 + m2);
          const int o = (l0 - m0 + P) + W * (l1 - m1 + P) + W * W * (l2 - m2 + P);
          a.bt[row * (W * W * W) + o] += val;
        }
      }
  }
}

template <int P>
constexpr int stiffness_3d_smem() {
  constexpr int NQ = P + 1, P1 = P + 1;
  return (NQ * NQ * NQ * 9 + 6 * NQ * P1 + 9 * NQ * NQ * P1 * P1) * (int)sizeof(double);
}

// band[idx[i]] += val[i] (indices distinct)
__global__ void band_add(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ val,
                         double* __restrict__ band) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) band[idx[i]] += val[i];
}

// band[o * nloc + r] = bt[r * nb + o], through 32 x 32 shared-memory tiles (both sides coalesced)
__global__ void band_transpose(int nb, int64_t nloc, const double* __restrict__ bt, double* __restrict__ band) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int o0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int64_t r = r0 + j;
    const int o = o0 + threadIdx.x;
    tile[j][threadIdx.x] = (r < nloc && o < nb) ? bt[r * nb + o] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int o = o0 + j;
    const int64_t r = r0 + threadIdx.x;
    if (o < nb && r < nloc) band[(int64_t)o * nloc + r] = tile[threadIdx.x][j];
  }
}

// strong Dirichlet condition: band entries whose row or column is a Dirichlet function are zeroed
// (columns leaving the patch are never written); band_off[k nb + o] = the position offset of o in patch k
__global__ void band_dirichlet(int nb, int64_t nloc, int K, const int64_t* __restrict__ off,
                               const int64_t* __restrict__ band_off, const unsigned char* __restrict__ dirichlet,
                               double* __restrict__ band) {
  const int o = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nloc) return;
  double* b = band + (int64_t)o * nloc + r;
  if (*b == 0.0) return;
  int k = 0;
  while (r >= off[k + 1]) ++k;
  const int64_t c = r + band_off[(int64_t)k * nb + o];
  if (dirichlet[r] || c < off[k] || c >= off[k + 1] || dirichlet[c]) *b = 0.0;
}

// One direction of the Galerkin product of a patch band (Sec. 3, Eq. a:galerkin): rows and offsets
// along `dir` go from fine to coarse, the other directions unchanged,
//   out[(I, rest), (O, o_rest)] = sum_{i, j} P[i, I] in[(i, rest), (j - i, o_rest)] P[j, I + O],
// children i of I from the transfer tables (ascending), zero coefficients skipped; one thread per
// output entry.  in / out: band[o * ld + r] of the patch (r the patch-local row)
struct GalArgs {
  const double* in;
  double* out;
  int64_t ld_in, ld_out;
  int nin[3], nout[3];
  int dir, p, nb, cw;
  const int* ch_start;    // coarse index -> first child (this patch and direction)
  const double* ch_val;   // coarse index x cw
};

__global__ void galerkin_dir(GalArgs g) {
  const int o = blockIdx.y;
  const int64_t rows_out = (int64_t)g.nout[0] * g.nout[1] * g.nout[2];
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows_out) return;
  const int W = 2 * g.p + 1;
  const int wpow[3] = {1, W, W * W};
  const int O = (o / wpow[g.dir]) % W - g.p;
  int idx[3];
  int64_t rem = r;
  for (int a = 0; a < 3; ++a) { idx[a] = (int)(rem % g.nout[a]); rem /= g.nout[a]; }
  const int I = idx[g.dir], J = I + O;
  double s = 0.0;
  if (J >= 0 && J < g.nout[g.dir]) {
    const int64_t fstride[3] = {1, g.nin[0], (int64_t)g.nin[0] * g.nin[1]};
    const int64_t fbase = idx[0] + fstride[1] * idx[1] + fstride[2] * idx[2] - fstride[g.dir] * I;
    const int cI = g.ch_start[I], cJ = g.ch_start[J];
    for (int t = 0; t < g.cw; ++t) {
      const double pi = g.ch_val[(int64_t)I * g.cw + t];
      if (pi == 0.0) continue;
      const int i = cI + t;
      const int64_t frow = fbase + fstride[g.dir] * i;
      for (int u = 0; u < g.cw; ++u) {
        const double pj = g.ch_val[(int64_t)J * g.cw + u];
        if (pj == 0.0) continue;
        const int od = cJ + u - i;
        if (od < -g.p || od > g.p) continue;
        const int ofine = o + (od - O) * wpow[g.dir];
        s += pi * g.in[(int64_t)ofine * g.ld_in + frow] * pj;
      }
    }
  }
  g.out[(int64_t)o * g.ld_out + r] = s;
}

template <int P>
void launch_stiffness(int dim, int nctas, cudaStream_t st, const AsmArgs& a) {
  if (nctas == 0) return;
  count_launch();
  if (dim == 2) {
    stiffness_2d<P><<<nctas, 128, 0, st>>>(a);
  } else {
    stiffness_3d<P><<<nctas, 256, stiffness_3d_smem<P>(), st>>>(a);
  }
}

template <int P>
void prepare_stiffness_3d() {
  SCK(cudaFuncSetAttribute(stiffness_3d<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, stiffness_3d_smem<P>()));
}

template <class T>
T* dalloc(size_t n, std::vector<void*>& temps, cudaStream_t st) {
  void* p = nullptr;
  SCK(cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), st));
  temps.push_back(p);
  return static_cast<T*>(p);
}

template <class T>
T* dupload(const std::vector<T>& v, std::vector<void*>& temps, cudaStream_t st) {
  T* p = dalloc<T>(v.size(), temps, st);
  if (!v.empty()) SCK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return p;
}

struct Temps {
  std::vector<void*> ptrs;
  cudaStream_t st;
  ~Temps() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
};

// position offset of band index o in patch k (the host's Level::band_offset)
std::vector<int64_t> band_offsets(const Level& L) {
  std::vector<int64_t> bo((size_t)L.K * L.nb);
  for (int k = 0; k < L.K; ++k)
    for (int o = 0; o < L.nb; ++o) bo[(size_t)k * L.nb + o] = L.band_offset(k, o);
  return bo;
}

void dirichlet_on_device(const Level& L, double* band, Temps& T) {
  if (L.nloc == 0) return;
  const int64_t* off = dupload(L.off, T.ptrs, T.st);
  const int64_t* bo = dupload(band_offsets(L), T.ptrs, T.st);
  const unsigned char* dir = dupload(L.dirichlet, T.ptrs, T.st);
  count_launch();
  band_dirichlet<<<dim3((unsigned)((L.nloc + 255) / 256), (unsigned)L.nb), 256, 0, T.st>>>(L.nb, L.nloc, L.K, off, bo,
                                                                                         dir, band);
}

}  // namespace

bool gpu_setup_supported(const Problem& pr) {
  return pr.p >= 1 && pr.p <= 6 && (pr.d == 2 || pr.d == 3);
}

void gpu_assemble_finest(const Problem& pr, Level& F, double* band, cudaStream_t st) {
  Temps T;
  T.st = st;
  const int d = pr.d, p = pr.p, P1 = p + 1, nq = p + 1;
  // quadrature and geometry tables, per patch and direction (host: 1D work only)
  std::vector<QTab> qt((size_t)F.K * 3);
  std::vector<int> span, gspan;
  std::vector<double> w, B, D, gB, gD;
  std::vector<PatchGeo> geo(F.K);
  std::vector<double> ctrl;
  int G1 = 1;
  for (int k = 0; k < F.K; ++k) G1 = std::max(G1, pr.geo[k].q + 1);
  double xg[16], wg[16];
  gauss_legendre(nq, xg, wg);
  for (int k = 0; k < F.K; ++k) {
    const Geometry& g = pr.geo[k];
    geo[k].ctrl = (int64_t)ctrl.size();  // in doubles
    for (int a = 0; a < 3; ++a) geo[k].ncp[a] = g.ncp[a];
    geo[k].q = g.q;
    ctrl.insert(ctrl.end(), g.ctrl.begin(), g.ctrl.end());
    for (int a = 0; a < 3; ++a) {
      QTab& q = qt[(size_t)k * 3 + a];
      q.e0 = (int64_t)span.size();
      q.q0 = (int64_t)w.size();
      if (a >= d) { q.ne = 1; continue; }
      const Vec& t = F.knots[k][a];
      const Vec z = breakpoints(t);
      q.ne = (int)z.size() - 1;
      double N[16], dN[16];
      for (int e = 0; e < q.ne; ++e) {
        const double lo = z[e], h = z[e + 1] - z[e];
        const int s = find_span(t, p, lo + 0.5 * h);
        span.push_back(s);
        for (int j = 0; j < nq; ++j) {
          const double x = lo + h * xg[j];
          w.push_back(h * wg[j]);
          basis_on_span(t, p, s, x, N, dN);
          for (int l = 0; l < P1; ++l) { B.push_back(N[l]); D.push_back(dN[l]); }
          const int gs = find_span(g.knots[a], g.q, x);
          gspan.push_back(gs);
          basis_on_span(g.knots[a], g.q, gs, x, N, dN);
          for (int l = 0; l < G1; ++l) { gB.push_back(l <= g.q ? N[l] : 0.0); gD.push_back(l <= g.q ? dN[l] : 0.0); }
        }
      }
    }
  }
  std::vector<PatchMeta> pm(F.K);
  for (int k = 0; k < F.K; ++k) {
    pm[k].off = F.off[k];
    for (int a = 0; a < 3; ++a) pm[k].N[a] = F.N[k][a];
  }
  AsmArgs a{};
  a.qt = dupload(qt, T.ptrs, st);
  a.span = dupload(span, T.ptrs, st);
  a.w = dupload(w, T.ptrs, st);
  a.B = dupload(B, T.ptrs, st);
  a.D = dupload(D, T.ptrs, st);
  a.gspan = dupload(gspan, T.ptrs, st);
  a.gB = dupload(gB, T.ptrs, st);
  a.gD = dupload(gD, T.ptrs, st);
  a.G1 = G1;
  a.geo = dupload(geo, T.ptrs, st);
  a.ctrl = dupload(ctrl, T.ptrs, st);
  a.pm = dupload(pm, T.ptrs, st);
  double* bt = dalloc<double>((size_t)F.nb * F.nloc, T.ptrs, st);
  a.bt = bt;
  a.nloc = F.nloc;
  // CTA prefixes of every colour (elements with index residues c modulo p + 1)
  const int ncol = d == 2 ? P1 * P1 : P1 * P1 * P1;
  std::vector<int> prefix((size_t)ncol * (F.K + 1), 0);
  for (int c = 0; c < ncol; ++c) {
    const int cc[3] = {c % P1, (c / P1) % P1, d == 3 ? c / (P1 * P1) : 0};
    for (int k = 0; k < F.K; ++k) {
      int64_t n = 1;
      for (int a2 = 0; a2 < d; ++a2) n *= std::max(0, (qt[(size_t)k * 3 + a2].ne - cc[a2] + P1 - 1) / P1);
      prefix[(size_t)c * (F.K + 1) + k + 1] = prefix[(size_t)c * (F.K + 1) + k] + (int)n;
    }
  }
  const int* dprefix = dupload(prefix, T.ptrs, st);
  if (d == 3) {
    switch (p) {
      case 1: prepare_stiffness_3d<1>(); break;
      case 2: prepare_stiffness_3d<2>(); break;
      case 3: prepare_stiffness_3d<3>(); break;
      case 4: prepare_stiffness_3d<4>(); break;
      case 5: prepare_stiffness_3d<5>(); break;
      default: prepare_stiffness_3d<6>(); break;
    }
  }
  SCK(cudaMemsetAsync(bt, 0, (size_t)F.nb * F.nloc * sizeof(double), st));
  for (int c = 0; c < ncol; ++c) {
    a.c0 = c % P1;
    a.c1 = (c / P1) % P1;
    a.c2 = d == 3 ? c / (P1 * P1) : 0;
    a.cta_ptr = dprefix + (size_t)c * (F.K + 1);
    const int nctas = prefix[(size_t)c * (F.K + 1) + F.K];
    switch (p) {
      case 1: launch_stiffness<1>(d, nctas, st, a); break;
      case 2: launch_stiffness<2>(d, nctas, st, a); break;
      case 3: launch_stiffness<3>(d, nctas, st, a); break;
      case 4: launch_stiffness<4>(d, nctas, st, a); break;
      case 5: launch_stiffness<5>(d, nctas, st, a); break;
      default: launch_stiffness<6>(d, nctas, st, a); break;
    }
    SCK(cudaGetLastError());
  }
  count_launch();
  band_transpose<<<dim3((unsigned)((F.nloc + 31) / 32), (unsigned)((F.nb + 31) / 32)), dim3(32, 8), 0, st>>>(
      F.nb, F.nloc, bt, band);
  SCK(cudaGetLastError());
  // the SIPG terms within one patch (host, in cell order): merged per band entry, then added
  if (!F.band_add.empty()) {
    std::vector<int64_t> idx;
    std::vector<double> val;
    for (const auto& x : F.merged_band_add()) { idx.push_back(x.first); val.push_back(x.second); }
    const int64_t* di = dupload(idx, T.ptrs, st);
    const double* dv = dupload(val, T.ptrs, st);
    count_launch();
    band_add<<<(unsigned)((idx.size() + 255) / 256), 256, 0, st>>>((int64_t)idx.size(), di, dv, band);
    SCK(cudaGetLastError());
    std::vector<std::pair<int64_t, double>>().swap(F.band_add);
  }
  dirichlet_on_device(F, band, T);
  SCK(cudaGetLastError());
  SCK(cudaStreamSynchronize(st));
}

void gpu_galerkin_band(const Level& Fl, const Level& C, const Transfer& Tr, const double* fband, double* cband,
                       cudaStream_t st) {
  Temps T;
  T.st = st;
  const int d = Fl.d, p = Fl.p, nb = Fl.nb;
  // children tables of every patch and direction: first child, cw values (zero padded)
  int cw = 1;
  for (int k = 0; k < Fl.K; ++k)
    for (int a = 0; a < d; ++a) {
      const int nf = Fl.N[k][a], nc = C.N[k][a];
      for (int I = 0; I < nc; ++I) {
        int lo = nf, hi = -1;
        for (int i = 0; i < nf; ++i)
          if (Tr.P[k][a][(size_t)i * nc + I] != 0.0) { lo = std::min(lo, i); hi = std::max(hi, i); }
        if (hi >= lo) cw = std::max(cw, hi - lo + 1);
      }
    }
  std::vector<int> cs;
  std::vector<double> cv;
  std::vector<int64_t> coff((size_t)Fl.K * 3, 0);
  for (int k = 0; k < Fl.K; ++k)
    for (int a = 0; a < d; ++a) {
      coff[(size_t)k * 3 + a] = (int64_t)cs.size();
      const int nf = Fl.N[k][a], nc = C.N[k][a];
      const Vec& P = Tr.P[k][a];
      for (int I = 0; I < nc; ++I) {
        int lo = 0;
        while (lo < nf && P[(size_t)lo * nc + I] == 0.0) ++lo;
        if (lo == nf) lo = 0;
        cs.push_back(lo);
        for (int t = 0; t < cw; ++t) cv.push_back(lo + t < nf ? P[(size_t)(lo + t) * nc + I] : 0.0);
      }
    }
  const int* dcs = dupload(cs, T.ptrs, st);
  const double* dcv = dupload(cv, T.ptrs, st);
  // intermediate bands: the largest patch after one and two directions
  int64_t tmax = 1;
  for (int k = 0; k < Fl.K; ++k) {
    std::array<int, 3> n = Fl.N[k];
    for (int a = 0; a + 1 < d; ++a) {
      n[a] = C.N[k][a];
      tmax = std::max<int64_t>(tmax, (int64_t)n[0] * n[1] * n[2]);
    }
  }
  double* t0 = dalloc<double>((size_t)nb * tmax, T.ptrs, st);
  double* t1 = d == 3 ? dalloc<double>((size_t)nb * tmax, T.ptrs, st) : nullptr;
  for (int k = 0; k < Fl.K; ++k) {
    GalArgs g{};
    g.p = p;
    g.nb = nb;
    g.cw = cw;
    std::array<int, 3> n = Fl.N[k];
    const double* in = fband + Fl.off[k];
    int64_t ld_in = Fl.nloc;
    for (int a = 0; a < d; ++a) {
      const bool last = a == d - 1;
      double* out = last ? cband + C.off[k] : (a == 0 ? t0 : t1);
      std::array<int, 3> nn = n;
      nn[a] = C.N[k][a];
      g.in = in;
      g.out = out;
      g.ld_in = ld_in;
      g.ld_out = last ? C.nloc : (int64_t)nn[0] * nn[1] * nn[2];
      for (int x = 0; x < 3; ++x) { g.nin[x] = n[x]; g.nout[x] = nn[x]; }
      g.dir = a;
      g.ch_start = dcs + coff[(size_t)k * 3 + a];
      g.ch_val = dcv + coff[(size_t)k * 3 + a] * cw;
      const int64_t rows = (int64_t)nn[0] * nn[1] * nn[2];
      count_launch();
      galerkin_dir<<<dim3((unsigned)((rows + 127) / 128), (unsigned)nb), 128, 0, st>>>(g);
      SCK(cudaGetLastError());
      in = out;
      ld_in = g.ld_out;
      n = nn;
    }
  }
  dirichlet_on_device(C, cband, T);
  SCK(cudaGetLastError());
  SCK(cudaStreamSynchronize(st));
}

}  // namespace dev
}  // namespace mgiga
