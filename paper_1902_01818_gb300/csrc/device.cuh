// Device-side data of libmgiga and the kernel launchers.
//
// Layout in HBM (one grid level):
//   * vectors: all patch blocks back to back (local layout), patch k holding
//     prod_a N_a coefficients with xi_0 fastest; Dirichlet entries are 0.
//     Each vector has a zero guard of `guard` doubles on both sides so that
//     band neighbours of boundary rows stay inside the allocation.
//   * operator: band[o * nloc + pos], o = sum_a (o_a + p)(2p+1)^a, the
//     coefficient coupling row pos to column pos + sum_a o_a stride_a of the
//     same patch (0 where that column leaves the patch or is Dirichlet);
//     consecutive rows are consecutive in memory, so a warp over rows reads
//     each offset's coefficients coalesced.
//   * SIPG cross-patch couplings in CSR over the rows that have them.
//   * conforming interfaces: DoFs shared by several patches are stored once
//     per patch; classes list their copies (owner first).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mgiga {
namespace dev {

constexpr int kTile = 256;  // rows per tile of the position-parallel kernels

struct PatchMeta {
  int64_t off;
  int N[3];
};

struct Tile {
  int patch;
  int count;
  int64_t start;
};

// per patch and direction: prolongation table between two levels
struct XferMeta {
  int64_t par_off;  // into par_start / par_val (fine index based)
  int64_t ch_off;   // into ch_start / ch_val (coarse index based)
  int nf, nc;
};

// C(m, n) = alpha * sum_k A(m, k) B(k, n) (+ epilogue) for one batched task.
// A is M x K: A[m * lda + k] (transA = 0) or A[k * lda + m] (transA = 1).
// B is K x N: B[k * ldb + n] (transB = 0) or B[n * ldb + k] (transB = 1).
// C[m * ldc + col(n)], col(n) = (n / ndiv) * nhi + n % ndiv (ndiv = N: plain);
// the split column lets C be the interior block of a 3D patch.
// batch z adds z * sA, z * sB, z * sC.  tA, tB, tC: element type of A, B, C
// (0 = double, 1 = float); the arithmetic type is the kernel's.
// epi 0: C = acc; 1: C = acc dinv[m ldd + n] (dinv: the inverse eigenvalue
//     sums of the fast diagonalisation, in the arithmetic type); 2: C += alpha acc.
struct GemmTask {
  int M, N, K, transA, transB, batch, ndiv, epi;
  const void* A;
  const void* B;
  void* C;
  int64_t lda, ldb, ldc, nhi, sA, sB, sC;
  double alpha;
  const void* dinv;
  int64_t ldd;
  int tA, tB, tC;
  // vec: A (transA 0) and B (transB 1) FP32, K contiguous, rows 16-byte aligned and zero beyond K
  // up to the next multiple of 4 (16-byte copies); ctrans: C[m][n] stored at n ldc + m
  int vec, ctrans;
};

struct GemmItem {
  int task, z, tm, tn;
};

struct PieceMeta {
  int64_t z_off;    // dense inverse n x n at zpool + z_off
  int64_t dof_off;  // primary positions at piece_pos + dof_off
  int n, pad;
};

struct PieceItem {
  int piece, row0;
};

// one 2D patch interior for the fused small fast diagonalisation: U_0 (n0 x
// n0), U_1 (n1 x n1) row-major and the inverse eigenvalue sums (n1 x n0) in
// the arithmetic type; the interior starts at ibase with row stride N0
struct FdSmall {
  int64_t ibase;
  int n0, n1, N0, pad;
  const void* U0;
  const void* U1;
  const void* dinv;
};

// one CTA of the fused 2D fast diagonalisation on the tensor cores (fd_fused_tf32): the
// 128 x 32 output tile (rb, cb) of  out = L (Rin Rt)  for one patch interior, where
//   pass 0:  Rin = R (interiors of r), Rt = U_0,   L = U_1^T,  out * dinv -> X (FP32)
//   pass 1:  Rin = X,                  Rt = U_0^T, L = U_1,    u_interior += tau out
// Every operand is FP32, row-major with its contraction index contiguous, rows 16-byte
// aligned and zero from the matrix width up to the pitch: rin[m * ldr + k] (n1 x n0),
// bt[n * ldb + k] = Rt(k, n) (n0 x n0), lm[m * ldl + k] = L(m, k) (n1 x n1).
struct FdFusedTask {
  const float* rin;
  const float* bt;
  const float* lm;
  const float* dinv;  // pass 0: n1 x n0, dinv[m * n0 + n]
  float* xout;        // pass 0: X[m * ldx + n], zero in the padding columns
  double* u;          // pass 1: u[ibase + m * N0 + n]
  int64_t ibase;
  int ldr, ldb, ldl, ldx, N0;
  int n0, n1, rb, cb, mt, pass;
};

// scalar slots of the CG state in device memory (S_TOL, S_NF, S_MAXIT: the parameters of a
// device-driven solve: tolerance, ||f||, iteration limit)
enum { S_RZ = 0, S_PQ, S_ALPHA, S_RR, S_RZNEW, S_BETA, S_FF, S_TMP, S_RZOLD, S_TOL, S_NF, S_MAXIT, S_COUNT };

// state of a device-driven PCG loop: iterations done, status (0 running, 1 converged, 2 iteration
// limit, 3 breakdown), the relative residual of the last iteration, executions of the confirming
// true residual and of the second half of an iteration
struct CgLoopState {
  int it, status, nconf, ncont;
  double rel;
};

}  // namespace dev
}  // namespace mgiga
