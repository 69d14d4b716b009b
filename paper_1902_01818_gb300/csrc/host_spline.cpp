// B-spline evaluation, quadrature, knot insertion, geometry and dense linear
// algebra for the set-up phase.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "host.hpp"

namespace mgiga {

int num_basis(const Vec& t, int p) { return (int)t.size() - p - 1; }

int find_span(const Vec& t, int p, double x) {
  const int n = num_basis(t, p);
  if (x >= t[n]) {  // right end point: last span of positive length
    int s = n - 1;
    while (s > p && t[s] == t[s + 1]) --s;
    return s;
  }
  if (x <= t[p]) {
    int s = p;
    while (s < n - 1 && t[s + 1] <= x) ++s;
    return s;
  }
  int lo = p, hi = n;  // invariant t[lo] <= x < t[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (x < t[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

// Triangular evaluation of the nonzero B-splines on span s (de Boor): the
// degree-j values are built from the degree-(j-1) values with the left and
// right distances x - t_{s+1-r} and t_{s+r} - x.
static void values_on_span(const Vec& t, int p, int s, double x, double* N) {
  double left[16], right[16];
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - t[s + 1 - j];
    right[j] = t[s + j] - x;
    double carry = 0.0;
    for (int r = 0; r < j; ++r) {
      const double den = right[r + 1] + left[j - r];
      const double q = den != 0.0 ? N[r] / den : 0.0;
      N[r] = carry + right[r + 1] * q;
      carry = left[j - r] * q;
    }
    N[j] = carry;
  }
}

void basis_on_span(const Vec& t, int p, int s, double x, double* N, double* dN) {
  values_on_span(t, p, s, x, N);
  if (!dN) return;
  if (p == 0) { dN[0] = 0.0; return; }
  double low[16];
  values_on_span(t, p - 1, s, x, low);  // functions s-p+1 .. s of degree p-1
  for (int r = 0; r <= p; ++r) {
    const int i = s - p + r;
    double a = 0.0, b = 0.0;
    if (r >= 1) {
      const double den = t[i + p] - t[i];
      if (den != 0.0) a = low[r - 1] / den;
    }
    if (r <= p - 1) {
      const double den = t[i + p + 1] - t[i + 1];
      if (den != 0.0) b = low[r] / den;
    }
    dN[r] = p * (a - b);
  }
}

Vec breakpoints(const Vec& t) {
  Vec z;
  for (double v : t)
    if (z.empty() || v > z.back()) z.push_back(v);
  return z;
}

Vec coarsen_knots(const Vec& t, int p) {
  const Vec z = breakpoints(t);
  const int n = (int)z.size() - 1;
  if (n % 2 != 0) throw SetupError(1, "cannot coarsen a knot vector with an odd number of intervals");
  Vec out(p + 1, z.front());
  for (int i = 2; i < n; i += 2) out.push_back(z[i]);
  for (int i = 0; i <= p; ++i) out.push_back(z.back());
  return out;
}

// Newton iteration on the Legendre polynomial P_m, evaluated by its
// three-term recurrence, from the Chebyshev-like start cos(pi (i + 3/4) / (m + 1/2)).
void gauss_legendre(int m, double* x, double* w) {
  for (int i = 0; i < m; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= m; ++j) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = m * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute the derivative at the converged node
    {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= m; ++j) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = m * (z * p0 - p1) / (z * z - 1.0);
    }
    // node on [-1,1] -> [0,1]; weight 2/((1-z^2) P'(z)^2) halved
    x[m - 1 - i] = 0.5 * (z + 1.0);
    w[m - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Boehm's algorithm: inserting knot x in span s replaces the coefficients
// c_{s-p+1..s} by convex combinations alpha c_i + (1 - alpha) c_{i-1},
// alpha = (x - t_i) / (t_{i+p} - t_i); coefficients before stay, after shift.
// Applied to all coarse basis functions at once (the columns of P).
Vec prolongation_1d(const Vec& tc, const Vec& tf, int p) {
  const int nc = num_basis(tc, p);
  const int nf = num_basis(tf, p);
  // knots of tf missing from tc (multiset difference)
  Vec ins;
  {
    size_t i = 0, j = 0;
    while (j < tf.size()) {
      if (i < tc.size() && tc[i] == tf[j]) { ++i; ++j; }
      else { ins.push_back(tf[j]); ++j; }
    }
    if (i != tc.size()) throw SetupError(1, "knot vectors are not nested");
  }
  Vec t = tc;
  std::vector<Vec> C(nc, Vec(nc, 0.0));  // C[i][j]: coefficient i of coarse function j
  for (int i = 0; i < nc; ++i) C[i][i] = 1.0;
  for (double x : ins) {
    const int n = (int)C.size();
    const int s = find_span(t, p, x);
    std::vector<Vec> D(n + 1, Vec(nc, 0.0));
    for (int i = 0; i <= n; ++i) {
      if (i <= s - p) D[i] = C[i];
      else if (i >= s + 1) D[i] = C[i - 1];
      else {
        const double alpha = (x - t[i]) / (t[i + p] - t[i]);
        for (int j = 0; j < nc; ++j) D[i][j] = alpha * C[i][j] + (1.0 - alpha) * C[i - 1][j];
      }
    }
    C.swap(D);
    t.insert(std::upper_bound(t.begin(), t.end(), x), x);
  }
  if ((int)C.size() != nf) throw SetupError(1, "knot insertion size mismatch");
  Vec P((size_t)nf * nc);
  for (int i = 0; i < nf; ++i)
    for (int j = 0; j < nc; ++j) P[(size_t)i * nc + j] = C[i][j];
  return P;
}

void param_matrices(const Vec& t, int p, Vec& K, Vec& M) {
  const int n = num_basis(t, p);
  K.assign((size_t)n * n, 0.0);
  M.assign((size_t)n * n, 0.0);
  const Vec z = breakpoints(t);
  double xg[16], wg[16], B[16], D[16];
  gauss_legendre(p + 1, xg, wg);
  for (size_t e = 0; e + 1 < z.size(); ++e) {
    const double a = z[e], h = z[e + 1] - z[e];
    const int s = find_span(t, p, a + 0.5 * h);
    for (int q = 0; q <= p; ++q) {
      const double x = a + h * xg[q], w = h * wg[q];
      basis_on_span(t, p, s, x, B, D);
      for (int r = 0; r <= p; ++r)
        for (int c = 0; c <= p; ++c) {
          const size_t idx = (size_t)(s - p + r) * n + (s - p + c);
          K[idx] += w * D[r] * D[c];
          M[idx] += w * B[r] * B[c];
        }
    }
  }
}

void geo_eval(const Problem& pr, int k, const double* xi, double* X, double* J) {
  const int d = pr.d;
  const Geometry& g = pr.geo[k];
  double B[3][16], D[3][16];
  int s[3];
  for (int a = 0; a < d; ++a) {
    s[a] = find_span(g.knots[a], g.q, xi[a]);
    basis_on_span(g.knots[a], g.q, s[a], xi[a], B[a], D[a]);
  }
  for (int c = 0; c < d; ++c) {
    X[c] = 0.0;
    for (int b = 0; b < d; ++b) J[c * d + b] = 0.0;
  }
  const int q1 = g.q + 1;
  const int n2 = d == 3 ? q1 : 1;
  for (int i2 = 0; i2 < n2; ++i2)
    for (int i1 = 0; i1 < q1; ++i1)
      for (int i0 = 0; i0 < q1; ++i0) {
        const int I0 = s[0] - g.q + i0, I1 = s[1] - g.q + i1;
        const int I2 = d == 3 ? s[2] - g.q + i2 : 0;
        const int64_t idx = I0 + (int64_t)g.ncp[0] * (I1 + (int64_t)g.ncp[1] * I2);
        const double* c = &g.ctrl[idx * d];
        double val = B[0][i0] * B[1][i1] * (d == 3 ? B[2][i2] : 1.0);
        double der[3];
        der[0] = D[0][i0] * B[1][i1] * (d == 3 ? B[2][i2] : 1.0);
        der[1] = B[0][i0] * D[1][i1] * (d == 3 ? B[2][i2] : 1.0);
        der[2] = d == 3 ? B[0][i0] * B[1][i1] * D[2][i2] : 0.0;
        for (int a = 0; a < d; ++a) {
          X[a] += val * c[a];
          for (int b = 0; b < d; ++b) J[a * d + b] += der[b] * c[a];
        }
      }
}

// ---------------------------------------------------------------------------
// dense linear algebra (row-major)
// ---------------------------------------------------------------------------

// Cholesky A = L L^T in place (lower triangle); false if a pivot is not
// positive.  Blocked left-looking: a panel of kChol columns is first updated
// with all earlier columns (row dot products, the panel's rows stay in cache),
// then factored column by column; rows run in parallel when `par`.
constexpr int kChol = 64;

// sum_k a[k] b[k] with eight independent partial sums (fixed order, vectorisable)
static inline double dot8(const double* a, const double* b, int n) {
  double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int k = 0;
  for (; k + 8 <= n; k += 8)
    for (int t = 0; t < 8; ++t) s[t] += a[k + t] * b[k + t];
  double r = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
  for (; k < n; ++k) r += a[k] * b[k];
  return r;
}

// Register tile of dot products: out[r][c] = sum_{k < n} a_r[k] b_c[k] for two
// rows a_r and four rows b_c, each entry as two-lane partial sums combined in a
// fixed order (GCC vector extension: 2 x f64 lanes on x86 and Arm alike).  Each
// loaded pair of values serves four (a) or two (b) products.
typedef double v2d __attribute__((vector_size(16)));

static inline v2d ld2(const double* p) {
  v2d v;
  std::memcpy(&v, p, sizeof(v));
  return v;
}

static inline void dot_2x4(const double* a0, const double* a1, const double* const b[4], int n, double out[2][4]) {
  v2d s0[4] = {}, s1[4] = {};
  int k = 0;
  for (; k + 2 <= n; k += 2) {
    const v2d x0 = ld2(a0 + k), x1 = ld2(a1 + k);
    const v2d y0 = ld2(b[0] + k), y1 = ld2(b[1] + k), y2 = ld2(b[2] + k), y3 = ld2(b[3] + k);
    s0[0] += x0 * y0; s0[1] += x0 * y1; s0[2] += x0 * y2; s0[3] += x0 * y3;
    s1[0] += x1 * y0; s1[1] += x1 * y1; s1[2] += x1 * y2; s1[3] += x1 * y3;
  }
  for (int c = 0; c < 4; ++c) {
    double t0 = s0[c][0] + s0[c][1], t1 = s1[c][0] + s1[c][1];
    if (k < n) {
      t0 += a0[k] * b[c][k];
      t1 += a1[k] * b[c][k];
    }
    out[0][c] = t0;
    out[1][c] = t1;
  }
}

static bool cholesky(Vec& A, int n, bool par = false) {
  bool ok = true;
  for (int jb = 0; jb < n && ok; jb += kChol) {
    const int je = std::min(n, jb + kChol);
    if (jb > 0) {
      // trailing update of the panel columns [jb, je): rows in pairs, columns in fours
      const int npair = (n - jb + 1) / 2;
#pragma omp parallel for schedule(static) if (par && n - jb > 128)
      for (int ip = 0; ip < npair; ++ip) {
        const int i = jb + 2 * ip;
        double* ri = &A[(size_t)i * n];
        double* ri1 = i + 1 < n ? &A[(size_t)(i + 1) * n] : nullptr;
        int j = jb;
        if (ri1)
          for (; j + 4 <= std::min(je, i + 1); j += 4) {  // every column of the tile <= i
            const double* b[4] = {&A[(size_t)j * n], &A[(size_t)(j + 1) * n], &A[(size_t)(j + 2) * n],
                                  &A[(size_t)(j + 3) * n]};
            double d[2][4];
            dot_2x4(ri, ri1, b, jb, d);
            for (int c = 0; c < 4; ++c) {
              ri[j + c] -= d[0][c];
              ri1[j + c] -= d[1][c];
            }
          }
        for (int jj = j; jj < std::min(je, i + 1); ++jj) ri[jj] -= dot8(ri, &A[(size_t)jj * n], jb);
        if (ri1)
          for (int jj = j; jj < std::min(je, i + 2); ++jj) ri1[jj] -= dot8(ri1, &A[(size_t)jj * n], jb);
      }
    }
    for (int j = jb; j < je; ++j) {
      double* rj = &A[(size_t)j * n];
      const double s = rj[j] - dot8(rj + jb, rj + jb, j - jb);
      if (!(s > 0.0)) { ok = false; break; }
      const double ljj = std::sqrt(s);
      rj[j] = ljj;
#pragma omp parallel for schedule(static) if (par && n - j > 256)
      for (int i = j + 1; i < n; ++i) {
        double* ri = &A[(size_t)i * n];
        ri[j] = (ri[j] - dot8(ri + jb, rj + jb, j - jb)) / ljj;
      }
    }
  }
  return ok;
}

// Wt = (L^{-1})^T for the lower-triangular L (row-major): row c of Wt is
// column c of L^{-1}, by forward substitution.  Columns are solved kInvCols at
// a time so that each row of L is read once per group (in parallel over
// groups when `par`); within a group four columns and two rows at a time (the
// entries of Wt before a column's diagonal are zero, so the four columns share
// the group's index range; the second row adds its term on the first after
// that row is solved).
constexpr int kInvCols = 64;

static Vec lower_inverse_t(const Vec& L, int n, bool par = false) {
  Vec Wt((size_t)n * n, 0.0);
  const int ngroups = (n + kInvCols - 1) / kInvCols;
#pragma omp parallel for schedule(dynamic) if (par && n > 256)
  for (int g = 0; g < ngroups; ++g) {
    const int c0 = g * kInvCols, c1 = std::min(n, c0 + kInvCols);
    int c = c0;
    for (; c + 4 <= c1; c += 4) {
      const double* b[4] = {&Wt[(size_t)c * n] + c, &Wt[(size_t)(c + 1) * n] + c, &Wt[(size_t)(c + 2) * n] + c,
                            &Wt[(size_t)(c + 3) * n] + c};
      double* w[4] = {&Wt[(size_t)c * n], &Wt[(size_t)(c + 1) * n], &Wt[(size_t)(c + 2) * n],
                      &Wt[(size_t)(c + 3) * n]};
      int i = c;
      for (; i + 2 <= n; i += 2) {
        const double* li = &L[(size_t)i * n];
        const double* li1 = &L[(size_t)(i + 1) * n];
        double d[2][4];
        dot_2x4(li + c, li1 + c, b, i - c, d);
        for (int q = 0; q < 4; ++q) {
          const int cq = c + q;
          const double wi = cq <= i ? ((i == cq ? 1.0 : 0.0) - d[0][q]) / li[i] : 0.0;
          w[q][i] = wi;
          if (cq <= i + 1) w[q][i + 1] = ((i + 1 == cq ? 1.0 : 0.0) - (d[1][q] + li1[i] * wi)) / li1[i + 1];
        }
      }
      for (; i < n; ++i) {
        const double* li = &L[(size_t)i * n];
        for (int q = 0; q < 4; ++q) {
          const int cq = c + q;
          if (cq > i) continue;
          w[q][i] = ((i == cq ? 1.0 : 0.0) - dot8(li + c, w[q] + c, i - c)) / li[i];
        }
      }
    }
    for (int i = c; i < n; ++i) {  // the group's last columns one at a time
      const double* li = &L[(size_t)i * n];
      for (int cc = c; cc < std::min(c1, i + 1); ++cc) {
        double* w = &Wt[(size_t)cc * n];
        w[i] = ((i == cc ? 1.0 : 0.0) - dot8(li + cc, w + cc, i - cc)) / li[i];
      }
    }
  }
  return Wt;
}

// A^{-1} = L^{-T} L^{-1} = W^T W for the SPD A; the factorisation and the
// products run in parallel (OpenMP) when `par` -- for large pieces processed
// one at a time
Vec spd_inverse(const Vec& A, int n, bool par) {
  Vec L = A;
  if (!cholesky(L, n, par)) throw SetupError(4, "Cholesky factorisation broke down (matrix not SPD)");
  const Vec Wt = lower_inverse_t(L, n, par);
  // Z[i][j] = sum_{k >= max(i, j)} Wt[i][k] Wt[j][k], j <= i; a block of kInvCols rows i stays
  // in cache while every row j is read once per block; rows in pairs and columns in fours where
  // the tile lies below the diagonal (Wt[i][k] = 0 for k < i, so the pair shares the range k >= i)
  Vec Z((size_t)n * n, 0.0);
  const int nblk = (n + kInvCols - 1) / kInvCols;
#pragma omp parallel for schedule(dynamic) if (par && n > 256)
  for (int bk = 0; bk < nblk; ++bk) {
    const int i0 = bk * kInvCols, i1 = std::min(n, i0 + kInvCols);
    for (int i = i0; i < i1; i += 2) {
      const bool two = i + 1 < i1;
      const double* wi = &Wt[(size_t)i * n];
      const double* wi1 = two ? &Wt[(size_t)(i + 1) * n] : nullptr;
      int j = 0;
      if (two)
        for (; j + 4 <= i + 1; j += 4) {  // columns j..j+3 <= i
          const double* b[4] = {&Wt[(size_t)j * n] + i, &Wt[(size_t)(j + 1) * n] + i,
                                &Wt[(size_t)(j + 2) * n] + i, &Wt[(size_t)(j + 3) * n] + i};
          double d[2][4];
          dot_2x4(wi + i, wi1 + i, b, n - i, d);
          for (int q = 0; q < 4; ++q) {
            Z[(size_t)i * n + j + q] = d[0][q];
            Z[(size_t)(j + q) * n + i] = d[0][q];
            Z[(size_t)(i + 1) * n + j + q] = d[1][q];
            Z[(size_t)(j + q) * n + i + 1] = d[1][q];
          }
        }
      for (int r = i; r < (two ? i + 2 : i + 1); ++r)
        for (int jj = j; jj <= r; ++jj) {
          const double v = dot8(&Wt[(size_t)r * n] + r, &Wt[(size_t)jj * n] + r, n - r);
          Z[(size_t)r * n + jj] = v;
          Z[(size_t)jj * n + r] = v;
        }
    }
  }
  return Z;
}

// Symmetric eigen-decomposition C = V diag(lam) V^T (C n x n, row-major; returns Vt = V^T,
// row j the eigenvector of lam[j]).  Householder reduction to tridiagonal form, then the
// implicit QL iteration with Wilkinson-type shifts on the tridiagonal (Golub & Van Loan,
// Matrix Computations, Sec. 8.3), its plane rotations applied to the reduction's orthogonal
// factor.  O(n^3) with a small constant, rows contiguous in every update.
static void sym_eig(Vec C, int n, Vec& Vt, Vec& lam) {
  std::vector<Vec> hv(n);
  std::vector<double> hbeta(n, 0.0);
  Vec w(n), p(n);
  for (int k = 0; k + 2 < n; ++k) {
    // x = C[k+1.., k] = C[k, k+1..] (symmetric)
    double* rk = &C[(size_t)k * n];
    double norm2 = 0.0;
    for (int i = k + 1; i < n; ++i) norm2 += rk[i] * rk[i];
    const double x0 = rk[k + 1];
    const double tail = norm2 - x0 * x0;
    if (tail <= 1e-300 * std::max(norm2, 1e-300)) continue;  // already tridiagonal in this column
    const double alpha = x0 >= 0.0 ? -std::sqrt(norm2) : std::sqrt(norm2);
    Vec& v = hv[k];
    v.assign(n, 0.0);
    for (int i = k + 1; i < n; ++i) v[i] = rk[i];
    v[k + 1] -= alpha;
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    const double beta = 2.0 / vv;
    hbeta[k] = beta;
    // trailing block A22 -= v w^T + w v^T with p = beta A22 v, w = p - (beta/2)(p.v) v
    for (int i = k + 1; i < n; ++i) {
      const double* ri = &C[(size_t)i * n];
      double t = 0.0;
      for (int j = k + 1; j < n; ++j) t += ri[j] * v[j];
      p[i] = beta * t;
    }
    double pv = 0.0;
    for (int i = k + 1; i < n; ++i) pv += p[i] * v[i];
    for (int i = k + 1; i < n; ++i) w[i] = p[i] - 0.5 * beta * pv * v[i];
    for (int i = k + 1; i < n; ++i) {
      double* ri = &C[(size_t)i * n];
      for (int j = k + 1; j < n; ++j) ri[j] -= v[i] * w[j] + w[i] * v[j];
    }
    for (int i = k + 2; i < n; ++i) C[(size_t)k * n + i] = C[(size_t)i * n + k] = 0.0;
    C[(size_t)k * n + k + 1] = C[(size_t)(k + 1) * n + k] = alpha;
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = C[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = C[(size_t)i * n + i + 1];
  // Vt = Q^T = H_{n-3} ... H_0: apply the reflections from the left to the identity
  Vt.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Vt[(size_t)i * n + i] = 1.0;
  for (int k = 0; k + 2 < n; ++k) {
    if (hbeta[k] == 0.0) continue;
    const Vec& v = hv[k];
    // Vt <- (I - beta v v^T) Vt: rows k+1..n-1 change
    std::fill(w.begin(), w.end(), 0.0);
    for (int i = k + 1; i < n; ++i) {
      const double* ri = &Vt[(size_t)i * n];
      const double vi = v[i];
      for (int j = 0; j < n; ++j) w[j] += vi * ri[j];
    }
    for (int i = k + 1; i < n; ++i) {
      double* ri = &Vt[(size_t)i * n];
      const double f = hbeta[k] * v[i];
      for (int j = 0; j < n; ++j) ri[j] -= f * w[j];
    }
  }
  // implicit QL on (d, e); rotations of rows i, i+1 of Vt
  const double eps = std::numeric_limits<double>::epsilon();
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m + 1 < n; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (iter >= 100) throw SetupError(4, "symmetric eigenvalue iteration did not converge");
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = m - 1;
      bool deflated = false;
      for (; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // split: the rotation would be undefined
          d[i + 1] -= pp;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        double* ra = &Vt[(size_t)i * n];
        double* rb = &Vt[(size_t)(i + 1) * n];
        for (int k = 0; k < n; ++k) {
          const double t = rb[k];
          rb[k] = s * ra[k] + c * t;
          ra[k] = c * ra[k] - s * t;
        }
      }
      if (deflated) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  lam.assign(d.begin(), d.end());
}

// Generalized symmetric-definite eigenproblem K U = M U diag(lam), U^T M U = I (M = L L^T):
// the symmetric C = L^{-1} K L^{-T} = V diag(lam) V^T, then U = L^{-T} V.
void gen_eig(const Vec& K, const Vec& M, int n, Vec& U, Vec& lam) {
  Vec L = M;
  if (!cholesky(L, n)) throw SetupError(4, "mass matrix not SPD");
  const Vec Wt = lower_inverse_t(L, n);  // row c: column c of W = L^{-1}
  // C = W K W^T with W = L^{-1} lower triangular (W[i][k] = Wt[k][i]); first T = W K
  Vec W((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) W[(size_t)i * n + j] = Wt[(size_t)j * n + i];
  Vec T((size_t)n * n, 0.0), C((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {  // T[i][:] = sum_{k <= i} W[i][k] K[k][:]
    double* ti = &T[(size_t)i * n];
    for (int k = 0; k <= i; ++k) {
      const double wik = W[(size_t)i * n + k];
      if (wik == 0.0) continue;
      const double* kk = &K[(size_t)k * n];
      for (int j = 0; j < n; ++j) ti[j] += wik * kk[j];
    }
  }
  for (int i = 0; i < n; ++i)  // C[i][j] = sum_{k <= j} T[i][k] W[j][k]
    for (int j = 0; j <= i; ++j) {
      const double* ti = &T[(size_t)i * n];
      const double* wj = &W[(size_t)j * n];
      double s = 0.0;
      for (int k = 0; k <= j; ++k) s += ti[k] * wj[k];
      C[(size_t)i * n + j] = s;
      C[(size_t)j * n + i] = s;
    }
  Vec Vt;
  sym_eig(C, n, Vt, lam);
  // U = W^T V: U[i][j] = sum_{k >= i} W[k][i] V[k][j] = sum_k Wt[i][k] Vt[j][k]
  U.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double* wi = &Wt[(size_t)i * n];
      const double* vj = &Vt[(size_t)j * n];
      double s = 0.0;
      for (int k = i; k < n; ++k) s += wi[k] * vj[k];
      U[(size_t)i * n + j] = s;
    }
}

}  // namespace mgiga
