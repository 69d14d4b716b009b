// Host-side set-up of libmgiga: B-splines, geometry, assembly, DoF topology,
// Galerkin hierarchy and smoother data.  Everything here runs once per
// problem (mgiga_create / mgiga_assemble); the solve itself runs on the GPU.
#pragma once

#include <array>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

namespace mgiga {

// Raised by the set-up code; the C entry points turn it into a status code.
struct SetupError : std::runtime_error {
  int status;
  SetupError(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

using Vec = std::vector<double>;

// ---------------------------------------------------------------------------
// B-splines on open knot vectors (Sec. 2, Eq. local)
// ---------------------------------------------------------------------------
int num_basis(const Vec& t, int p);
// span s with t[s] <= x < t[s+1], p <= s <= n-1; x at the right end -> last
// non-empty span
int find_span(const Vec& t, int p, double x);
// values (and first derivatives if dN != nullptr) of the p+1 B-splines
// s-p..s that are nonzero on span s, at x
void basis_on_span(const Vec& t, int p, int s, double x, double* N, double* dN);
Vec breakpoints(const Vec& t);
Vec coarsen_knots(const Vec& t, int p);
// m-point Gauss-Legendre rule on [0, 1]
void gauss_legendre(int m, double* x, double* w);
// prolongation from knots tc to tf (nested), dense row-major Nf x Nc, by
// Boehm knot insertion
Vec prolongation_1d(const Vec& tc, const Vec& tf, int p);
// 1D stiffness and mass on (0, 1), dense row-major N x N
void param_matrices(const Vec& t, int p, Vec& K, Vec& M);

// ---------------------------------------------------------------------------
// Problem and geometry
// ---------------------------------------------------------------------------
struct Geometry {
  int q = 1;
  std::array<Vec, 3> knots;
  std::array<int, 3> ncp{{1, 1, 1}};
  Vec ctrl;  // prod(ncp) * d, xi_0 fastest
};

struct Interface {
  int pa, sa, pb, sb;
  unsigned orient;
};

struct Problem {
  int d = 2, K = 0, p = 1;  // p: the largest patch degree (the reach of the patch band)
  std::vector<int> pk;      // degree of every patch (all p unless the problem lists one per patch)
  int deg(int k) const { return pk.empty() ? p : pk[k]; }
  std::vector<std::array<Vec, 3>> knots;  // finest level
  std::vector<Geometry> geo;
  std::vector<Interface> ifaces;
  int coupling = 0;
  double penalty = 0.0;
};

// X[d] and J[d*d] (J[a*d + b] = dX_a / dxi_b) at parameter xi[d]
void geo_eval(const Problem& pr, int k, const double* xi, double* X, double* J);

// ---------------------------------------------------------------------------
// One grid level: layout, numbering, operator
// ---------------------------------------------------------------------------
struct Level {
  int d = 2, p = 1, K = 0;  // p: the largest patch degree; band offsets span -p .. p
  std::vector<int> pk;      // degree of every patch
  int deg(int k) const { return pk.empty() ? p : pk[k]; }
  std::vector<std::array<Vec, 3>> knots;
  std::vector<std::array<int, 3>> N;  // B-splines per direction (unused dirs: 1)
  std::vector<int64_t> off;           // patch block offsets, K + 1 entries
  int64_t nloc = 0;                   // local layout length
  std::vector<int> patch_of;          // nloc: patch of a position
  std::vector<int> loc2glob;          // nloc: global DoF or -1 (Dirichlet)
  std::vector<uint8_t> dirichlet;     // nloc
  int ndof = 0;
  std::vector<int64_t> owner;         // ndof: position of the owning copy
  // conforming: classes of >= 2 copies, owner first
  std::vector<int> sh_ptr;            // nclass + 1
  std::vector<int64_t> sh_pos;
  Vec weight;                         // nloc: 1 / multiplicity (conforming)
  // operator: band[o * nloc + pos], o = sum_a (o_a + p) (2p+1)^a
  int nb = 0;
  Vec band;
  // the SIPG terms within one patch, (band index, value) in cell order, as the finest-level
  // assembly computes them (also added to the host band when there is one): the device set-up adds
  // them to the band it assembles, the matrix-free residual applies them as stored couplings
  std::vector<std::pair<int64_t, double>> band_add;
  bool record_band_add = false;  // list the within-patch SIPG terms also when a host band is assembled
  // the entries of band_add with equal band index summed in their listed (cell) order, by index
  std::vector<std::pair<int64_t, double>> merged_band_add() const;
  double nnz = 0.0;  // nonzero band coefficients (kept when the host band is released)
  // SIPG cross-patch couplings, CSR over rows x_row[i]
  std::vector<int64_t> x_row;
  std::vector<int> x_ptr;
  std::vector<int64_t> x_col;
  Vec x_val;

  int64_t pos(int k, int i0, int i1, int i2) const {
    return off[k] + i0 + (int64_t)N[k][0] * (i1 + (int64_t)N[k][1] * i2);
  }
  int64_t stride(int k, int a) const {
    return a == 0 ? 1 : a == 1 ? N[k][0] : (int64_t)N[k][0] * N[k][1];
  }
  int64_t band_offset(int k, int o) const;  // position offset of band index o
};

// numbering / topology of a level from its knots
void build_topology(const Problem& pr, Level& L);
// finest-level assembly: patch stiffness + SIPG interface terms into L.band / x-blocks (the terms
// within one patch also listed in L.band_add); with stiffness = false only the interface terms
// (L.band stays empty, the band being assembled on the GPU)
void assemble_fine(const Problem& pr, Level& L, const std::vector<std::array<Vec, 3>>& fine_knots,
                   bool stiffness = true);
// zero Dirichlet rows and columns of the band (when present on the host) and of the cross blocks
void apply_dirichlet(Level& L);
// load vector in global order
void assemble_load(const Problem& pr, const Level& L, double (*f)(const double*, void*), void* ctx,
                   double* out);

// prolongation data between level c (coarse) and f (fine): per patch and
// direction the dense 1D matrix Nf x Nc
struct Transfer {
  std::vector<std::array<Vec, 3>> P;  // per patch, per direction
};
Transfer build_transfer(const Level& C, const Level& F);
// Galerkin coarse operator A_c = P^T A_f P (band and cross blocks; band = false: the cross blocks
// only, the band being formed on the GPU)
void galerkin(const Level& F, const Transfer& T, Level& C, bool band = true);

// ---------------------------------------------------------------------------
// Smoother data
// ---------------------------------------------------------------------------
struct Piece {
  int kind;                  // 0 interior, 1 interface
  int patch;                 // interior: its patch
  std::vector<int> dofs;     // global DoFs, increasing
};
std::vector<Piece> decompose(const Problem& pr, const Level& L);

// interior fast diagonalisation data of one patch: U_a (n_a x n_a row-major,
// columns are M^-orthonormal eigenvectors), lambda_a, sigma
struct FDData {
  std::array<int, 3> n{{1, 1, 1}};
  std::array<Vec, 3> U, lam;
  double sigma = 0.0;
};
FDData fd_setup(const Level& L, int k, double delta);

// dense matrix of A restricted to the given global DoFs (row-major)
Vec restrict_dense(const Level& L, const std::vector<int>& dofs);
// inverse of an SPD matrix through its Cholesky factor (throws ENOTSPD)
// A^{-1} of the SPD n x n A (row-major); `par`: OpenMP inside (one large matrix at a time)
Vec spd_inverse(const Vec& A, int n, bool par = false);
// generalised eigenproblem K u = lambda M u, M SPD; U^T M U = I
void gen_eig(const Vec& K, const Vec& M, int n, Vec& U, Vec& lam);

std::vector<int> patch_parity(const Problem& pr);
std::vector<int> colouring(const Problem& pr, const Level& L);

// number of levels by the automatic rule
int auto_levels(const Problem& pr);

}  // namespace mgiga
