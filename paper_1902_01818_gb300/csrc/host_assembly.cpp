// DoF topology and assembly of the finest-level operator (Sec. 2 and 3).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>

#include <omp.h>

#include "host.hpp"

namespace mgiga {

int64_t Level::band_offset(int k, int o) const {
  int64_t off = 0;
  const int w = 2 * p + 1;
  for (int a = 0; a < d; ++a) {
    const int oa = o % w - p;
    o /= w;
    off += oa * stride(k, a);
  }
  return off;
}

static std::vector<int> tangential(int d, int side) {
  std::vector<int> t;
  for (int a = 0; a < d; ++a)
    if (a != side / 2) t.push_back(a);
  return t;
}

// ---------------------------------------------------------------------------
// numbering (Sec. 2, Eq. igaspace0: shared DoFs on matching interfaces;
// Sec. 3, Eq. igaspace: independent patches); Dirichlet DoFs are the ones
// with a nonzero trace on a side listed in no interface
// ---------------------------------------------------------------------------
namespace {
struct DSU {
  std::vector<int64_t> par;
  explicit DSU(int64_t n) : par(n) { std::iota(par.begin(), par.end(), 0); }
  int64_t find(int64_t x) {
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
  }
  void unite(int64_t a, int64_t b) {
    a = find(a); b = find(b);
    if (a == b) return;
    if (a < b) par[b] = a; else par[a] = b;
  }
};
}  // namespace

void build_topology(const Problem& pr, Level& L) {
  const int d = pr.d, K = pr.K, p = pr.p;
  L.d = d; L.p = p; L.K = K;
  L.pk.assign(K, p);
  for (int k = 0; k < K; ++k) L.pk[k] = pr.deg(k);
  L.N.assign(K, {{1, 1, 1}});
  L.off.assign(K + 1, 0);
  for (int k = 0; k < K; ++k) {
    int64_t sz = 1;
    for (int a = 0; a < d; ++a) {
      L.N[k][a] = num_basis(L.knots[k][a], pr.deg(k));
      sz *= L.N[k][a];
    }
    L.off[k + 1] = L.off[k] + sz;
  }
  L.nloc = L.off[K];
  L.patch_of.assign(L.nloc, 0);
  for (int k = 0; k < K; ++k)
    for (int64_t i = L.off[k]; i < L.off[k + 1]; ++i) L.patch_of[i] = k;

  // sides listed in interfaces
  std::vector<std::array<bool, 6>> iside(K);
  for (auto& s : iside) s.fill(false);
  for (const auto& f : pr.ifaces) { iside[f.pa][f.sa] = true; iside[f.pb][f.sb] = true; }
  L.dirichlet.assign(L.nloc, 0);
  for (int k = 0; k < K; ++k) {
    const auto& N = L.N[k];
    for (int i2 = 0; i2 < (d == 3 ? N[2] : 1); ++i2)
      for (int i1 = 0; i1 < N[1]; ++i1)
        for (int i0 = 0; i0 < N[0]; ++i0) {
          const int idx[3] = {i0, i1, i2};
          bool dir = false;
          for (int a = 0; a < d; ++a) {
            if (idx[a] == 0 && !iside[k][2 * a]) dir = true;
            if (idx[a] == N[a] - 1 && !iside[k][2 * a + 1]) dir = true;
          }
          L.dirichlet[L.pos(k, i0, i1, i2)] = dir;
        }
  }

  DSU dsu(L.nloc);
  const bool conforming = pr.coupling == 0;
  if (conforming) {
    for (const auto& f : pr.ifaces) {
      const auto ta = tangential(d, f.sa), tb = tangential(d, f.sb);
      const auto& Na = L.N[f.pa];
      const auto& Nb = L.N[f.pb];
      const int m = d - 1;
      const int n0 = Na[ta[0]], n1 = m == 2 ? Na[ta[1]] : 1;
      for (int j1 = 0; j1 < n1; ++j1)
        for (int j0 = 0; j0 < n0; ++j0) {
          int ia[3], ib[3];
          ia[f.sa / 2] = f.sa % 2 ? Na[f.sa / 2] - 1 : 0;
          ia[ta[0]] = j0;
          if (m == 2) ia[ta[1]] = j1;
          int tbm[2] = {j0, j1};
          if (m == 2 && (f.orient & 4u)) std::swap(tbm[0], tbm[1]);
          for (int c = 0; c < m; ++c)
            if (f.orient & (1u << c)) tbm[c] = Nb[tb[c]] - 1 - tbm[c];
          ib[f.sb / 2] = f.sb % 2 ? Nb[f.sb / 2] - 1 : 0;
          for (int c = 0; c < m; ++c) ib[tb[c]] = tbm[c];
          if (d == 2) { ia[2] = 0; ib[2] = 0; }
          for (int c = 0; c < m; ++c)
            if (tbm[c] < 0 || tbm[c] >= Nb[tb[c]]) throw SetupError(1, "interface knots do not match");
          if (Na[ta[0]] != Nb[tb[(m == 2 && (f.orient & 4u)) ? 1 : 0]])
            throw SetupError(1, "conforming interface with different numbers of B-splines");
          dsu.unite(L.pos(f.pa, ia[0], ia[1], ia[2]), L.pos(f.pb, ib[0], ib[1], ib[2]));
        }
    }
  }
  // a class is Dirichlet if any copy is
  std::vector<uint8_t> root_dir(L.nloc, 0);
  std::vector<int64_t> root(L.nloc);
  for (int64_t i = 0; i < L.nloc; ++i) {
    root[i] = conforming ? dsu.find(i) : i;
    if (L.dirichlet[i]) root_dir[root[i]] = 1;
  }
  L.loc2glob.assign(L.nloc, -1);
  L.owner.clear();
  std::vector<int> glob_of_root(L.nloc, -1);
  for (int64_t i = 0; i < L.nloc; ++i) {
    const int64_t r = root[i];
    if (root_dir[r]) { L.dirichlet[i] = 1; continue; }
    if (glob_of_root[r] < 0) {
      glob_of_root[r] = (int)L.owner.size();
      L.owner.push_back(i);
    }
    L.loc2glob[i] = glob_of_root[r];
  }
  L.ndof = (int)L.owner.size();
  // shared classes (conforming): owner first, then further copies ascending
  L.sh_ptr.assign(1, 0);
  L.sh_pos.clear();
  L.weight.assign(L.nloc, 1.0);
  if (conforming) {
    std::vector<int> count(L.ndof, 0);
    for (int64_t i = 0; i < L.nloc; ++i)
      if (L.loc2glob[i] >= 0) count[L.loc2glob[i]]++;
    std::vector<std::vector<int64_t>> copies;
    std::vector<int> cls(L.ndof, -1);
    for (int64_t i = 0; i < L.nloc; ++i) {
      const int g = L.loc2glob[i];
      if (g < 0) continue;
      L.weight[i] = 1.0 / count[g];
      if (count[g] < 2) continue;
      if (cls[g] < 0) { cls[g] = (int)copies.size(); copies.emplace_back(); }
      copies[cls[g]].push_back(i);
    }
    for (auto& c : copies) {
      for (int64_t x : c) L.sh_pos.push_back(x);
      L.sh_ptr.push_back((int)L.sh_pos.size());
    }
  }
}

// ---------------------------------------------------------------------------
// patch stiffness (Sec. 2): K_ij = sum_q w_q |det J| (J^{-T} grad^ B_i).(J^{-T} grad^ B_j),
// p+1 Gauss points per element and direction, sum-factorised over directions
// ---------------------------------------------------------------------------
namespace {
struct DirQuad {
  std::vector<int> span;        // per element
  std::vector<double> x, w;     // per element * nq
  std::vector<double> B, D;     // per element * nq * (p+1)
};

DirQuad dir_quad(const Vec& t, int p) {
  DirQuad q;
  const int nq = p + 1;
  const Vec z = breakpoints(t);
  double xg[16], wg[16];
  gauss_legendre(nq, xg, wg);
  const int ne = (int)z.size() - 1;
  q.span.resize(ne);
  q.x.resize((size_t)ne * nq);
  q.w.resize((size_t)ne * nq);
  q.B.resize((size_t)ne * nq * (p + 1));
  q.D.resize((size_t)ne * nq * (p + 1));
  for (int e = 0; e < ne; ++e) {
    const double a = z[e], h = z[e + 1] - z[e];
    q.span[e] = find_span(t, p, a + 0.5 * h);
    for (int k = 0; k < nq; ++k) {
      const double x = a + h * xg[k];
      q.x[(size_t)e * nq + k] = x;
      q.w[(size_t)e * nq + k] = h * wg[k];
      basis_on_span(t, p, q.span[e], x, &q.B[((size_t)e * nq + k) * (p + 1)],
                    &q.D[((size_t)e * nq + k) * (p + 1)]);
    }
  }
  return q;
}

// invert a d x d matrix (d = 2, 3); returns det
double inv_small(const double* J, int d, double* Ji) {
  if (d == 2) {
    const double det = J[0] * J[3] - J[1] * J[2];
    Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
    return det;
  }
  const double c00 = J[4] * J[8] - J[5] * J[7];
  const double c01 = J[5] * J[6] - J[3] * J[8];
  const double c02 = J[3] * J[7] - J[4] * J[6];
  const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  Ji[0] = c00 / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det; Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = c01 / det; Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = c02 / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det; Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  return det;
}
}  // namespace

static void patch_stiffness(const Problem& pr, Level& L, int k) {
  // p: this patch's degree (its basis and quadrature); the band spans offsets -pr.p .. pr.p
  const int d = pr.d, p = pr.deg(k), P1 = p + 1, nq = p + 1, W = 2 * pr.p + 1;
  DirQuad dq[3];
  int ne[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) { dq[a] = dir_quad(L.knots[k][a], p); ne[a] = (int)dq[a].span.size(); }
  const int slow = d - 1;
  const int Q = d == 2 ? nq * nq : nq * nq * nq;
  // the patch's band accumulated row-major (a row's offsets contiguous, so an
  // element's entries of one row share cache lines), stored offset-major at the end
  const int nb = L.nb;
  const int64_t off = L.off[k], rows = L.off[k + 1] - L.off[k];
  Vec Bt((size_t)rows * nb, 0.0);
  // band offset of entry (l, m) of an element matrix: ocode[m] - ocode[l] + ocode0, with
  // ocode[x] = x0 + W x1 + W^2 x2 for the local index x = x0 + P1 (x1 + P1 x2)
  std::vector<int> ocode(d == 2 ? P1 * P1 : P1 * P1 * P1);
  for (int x = 0; x < (int)ocode.size(); ++x)
    ocode[x] = x % P1 + W * ((x / P1) % P1) + (d == 3 ? W * W * (x / (P1 * P1)) : 0);
  const int ocode0 = pr.p + W * pr.p + (d == 3 ? W * W * pr.p : 0);
  // element slabs along the slowest direction touch disjoint band rows when
  // they are p+1 apart: p+1 parallel phases
  // (in 3D the rows of elements along xi_0 are coloured by both outer indices
  // modulo p+1: (p+1)^2 phases of many independent rows, enough for every core)
  const int nphase = d == 3 ? P1 * P1 : P1;
  for (int phase = 0; phase < nphase; ++phase) {
    const int r_slow = d == 3 ? phase / P1 : phase, r_mid = d == 3 ? phase % P1 : 0;
    const int n_slow = (ne[slow] - r_slow + P1 - 1) / P1;
    const int n_mid = d == 3 ? (ne[1] - r_mid + P1 - 1) / P1 : 1;
#pragma omp parallel
    {
      std::vector<double> C((size_t)Q * 9), T2, Ke;
      const int L2 = P1 * P1;
      T2.resize((size_t)9 * nq * nq * L2);  // 3D: the q2-contracted factors
      Ke.resize((size_t)(d == 2 ? L2 * L2 : L2 * L2 * L2));
#pragma omp for schedule(dynamic)
      for (int task = 0; task < n_slow * n_mid; ++task) {
        const int es = r_slow + P1 * (task / n_mid);
        const int e1m = r_mid + P1 * (task % n_mid);
          for (int e0 = 0; e0 < ne[0]; ++e0) {
            int e[3];
            e[0] = e0;
            if (d == 2) { e[1] = es; e[2] = 0; } else { e[1] = e1m; e[2] = es; }
            // geometric factors C_ab(q) = w |det J| (J^{-1} J^{-T})_ab
            for (int q2 = 0; q2 < (d == 3 ? nq : 1); ++q2)
              for (int q1 = 0; q1 < nq; ++q1)
                for (int q0 = 0; q0 < nq; ++q0) {
                  const int qi[3] = {q0, q1, q2};
                  double xi[3], w = 1.0;
                  for (int a = 0; a < d; ++a) {
                    xi[a] = dq[a].x[(size_t)e[a] * nq + qi[a]];
                    w *= dq[a].w[(size_t)e[a] * nq + qi[a]];
                  }
                  double X[3], J[9], Ji[9];
                  geo_eval(pr, k, xi, X, J);
                  const double det = inv_small(J, d, Ji);
                  const double s = w * std::fabs(det);
                  const int qq = q0 + nq * (q1 + nq * q2);
                  for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b) {
                      double v = 0.0;
                      for (int c = 0; c < d; ++c) v += Ji[a * d + c] * Ji[b * d + c];
                      C[(size_t)qq * 9 + a * 3 + b] = s * v;
                    }
                }
            std::fill(Ke.begin(), Ke.end(), 0.0);
            if (d == 2) {
              // Ke(l0 + P1 l1, m0 + P1 m1) = sum_q0 sum_ab X0_a(l0) X0_b(m0) U_ab(q0, l1, m1),
              // U_ab(q0, l1, m1) = sum_q1 C_ab(q0, q1) X1_a(l1) X1_b(m1), X_a the derivative along
              // direction a, else the value; C is symmetric, so only blocks l1 <= m1 are summed and
              // their transposes copied
              const double* V0 = &dq[0].B[(size_t)e[0] * nq * P1];  // [q][l]
              const double* D0 = &dq[0].D[(size_t)e[0] * nq * P1];
              const double* V1 = &dq[1].B[(size_t)e[1] * nq * P1];
              const double* D1 = &dq[1].D[(size_t)e[1] * nq * P1];
              double blk[16 * 16], h0[16], h1[16];
              for (int l1 = 0; l1 < P1; ++l1)
                for (int m1 = l1; m1 < P1; ++m1) {
                  for (int x = 0; x < P1 * P1; ++x) blk[x] = 0.0;
                  for (int q0 = 0; q0 < nq; ++q0) {
                    double u00 = 0.0, u01 = 0.0, u10 = 0.0, u11 = 0.0;
                    for (int q1 = 0; q1 < nq; ++q1) {
                      const double* c = &C[(size_t)(q0 + nq * q1) * 9];
                      const double va = V1[q1 * P1 + l1], da = D1[q1 * P1 + l1];
                      const double vb = V1[q1 * P1 + m1], db = D1[q1 * P1 + m1];
                      u00 += c[0] * va * vb;
                      u01 += c[1] * va * db;
                      u10 += c[3] * da * vb;
                      u11 += c[4] * da * db;
                    }
                    const double* g0 = &D0[q0 * P1];  // a = 0: derivative along xi_0
                    const double* g1 = &V0[q0 * P1];
                    for (int m0 = 0; m0 < P1; ++m0) {
                      h0[m0] = u00 * g0[m0] + u01 * g1[m0];
                      h1[m0] = u10 * g0[m0] + u11 * g1[m0];
                    }
                    for (int l0 = 0; l0 < P1; ++l0) {
                      const double a0 = g0[l0], a1 = g1[l0];
                      double* row = &blk[l0 * P1];
                      for (int m0 = 0; m0 < P1; ++m0) row[m0] += a0 * h0[m0] + a1 * h1[m0];
                    }
                  }
                  for (int l0 = 0; l0 < P1; ++l0)
                    for (int m0 = (l1 == m1 ? l0 : 0); m0 < P1; ++m0) {  // a diagonal block: its upper half
                      const double v = blk[l0 * P1 + m0];
                      Ke[(size_t)(l0 + P1 * l1) * L2 + (m0 + P1 * m1)] = v;
                      Ke[(size_t)(m0 + P1 * m1) * L2 + (l0 + P1 * l1)] = v;
                    }
                }
            } else {
              // Ke(l, m) = sum_q sum_ab C_ab(q) prod_dir X_dir,a(l_dir) X_dir,b(m_dir), X_dir,a the
              // derivative if a == dir, else the value.  Contract q2 (U), then per pair of row/column
              // indices (l1, l2), (m1, m2) with l1 + P1 l2 <= m1 + P1 m2 contract q1 (V); along xi_0
              // only "a == 0 or not" matters, so the nine pairs merge into a 2x2 form per q0 point
              const int L3 = L2 * P1;
              const double* Vd[3];
              const double* Dd[3];
              for (int dir = 0; dir < 3; ++dir) {
                Vd[dir] = &dq[dir].B[(size_t)e[dir] * nq * P1];  // [q][l]
                Dd[dir] = &dq[dir].D[(size_t)e[dir] * nq * P1];
              }
              // U[((ab * nq + q0) * nq + q1) * L2 + l2 * P1 + m2] = sum_q2 C_ab X2_a(l2) X2_b(m2)
              for (int ab = 0; ab < 9; ++ab) {
                const int aa = ab / 3, bb = ab % 3;
                const double* xa = aa == 2 ? Dd[2] : Vd[2];
                const double* xb = bb == 2 ? Dd[2] : Vd[2];
                for (int q0 = 0; q0 < nq; ++q0)
                  for (int q1 = 0; q1 < nq; ++q1) {
                    double* u = &T2[(((size_t)ab * nq + q0) * nq + q1) * L2];
                    for (int x = 0; x < L2; ++x) u[x] = 0.0;
                    for (int q2 = 0; q2 < nq; ++q2) {
                      const double c = C[(size_t)(q0 + nq * (q1 + nq * q2)) * 9 + aa * 3 + bb];
                      for (int l2 = 0; l2 < P1; ++l2) {
                        const double cl = c * xa[q2 * P1 + l2];
                        for (int m2 = 0; m2 < P1; ++m2) u[l2 * P1 + m2] += cl * xb[q2 * P1 + m2];
                      }
                    }
                  }
              }
              double blk[16 * 16], h0[16], h1[16];
              for (int L12 = 0; L12 < L2; ++L12)
                for (int M12 = L12; M12 < L2; ++M12) {
                  const int l1 = L12 % P1, l2 = L12 / P1, m1 = M12 % P1, m2 = M12 / P1;
                  for (int x = 0; x < P1 * P1; ++x) blk[x] = 0.0;
                  for (int q0 = 0; q0 < nq; ++q0) {
                    double v[9];
                    for (int ab = 0; ab < 9; ++ab) {
                      const int aa = ab / 3, bb = ab % 3;
                      const double* xa = aa == 1 ? Dd[1] : Vd[1];
                      const double* xb = bb == 1 ? Dd[1] : Vd[1];
                      const double* u = &T2[((size_t)ab * nq + q0) * nq * L2 + l2 * P1 + m2];
                      double t = 0.0;
                      for (int q1 = 0; q1 < nq; ++q1) t += u[(size_t)q1 * L2] * xa[q1 * P1 + l1] * xb[q1 * P1 + m1];
                      v[ab] = t;
                    }
                    const double w00 = v[0], w01 = v[1] + v[2], w10 = v[3] + v[6];
                    const double w11 = (v[4] + v[5]) + (v[7] + v[8]);
                    const double* g0 = &Dd[0][q0 * P1];  // a == 0: derivative along xi_0
                    const double* g1 = &Vd[0][q0 * P1];
                    for (int m0 = 0; m0 < P1; ++m0) {
                      h0[m0] = w00 * g0[m0] + w01 * g1[m0];
                      h1[m0] = w10 * g0[m0] + w11 * g1[m0];
                    }
                    for (int l0 = 0; l0 < P1; ++l0) {
                      const double a0 = g0[l0], a1 = g1[l0];
                      double* row = &blk[l0 * P1];
                      for (int m0 = 0; m0 < P1; ++m0) row[m0] += a0 * h0[m0] + a1 * h1[m0];
                    }
                  }
                  for (int l0 = 0; l0 < P1; ++l0)
                    for (int m0 = (L12 == M12 ? l0 : 0); m0 < P1; ++m0) {  // a diagonal block: its upper half
                      const double val = blk[l0 * P1 + m0];
                      Ke[(size_t)(l0 + P1 * L12) * L3 + (m0 + P1 * M12)] = val;
                      Ke[(size_t)(m0 + P1 * M12) * L3 + (l0 + P1 * L12)] = val;
                    }
                }
            }
            // scatter into the band: row of l, offset m - l
            const int LL = d == 2 ? L2 : L2 * P1;
            for (int l = 0; l < LL; ++l) {
              const int l0 = l % P1, l1 = (l / P1) % P1, l2 = l / (P1 * P1);
              const int r0 = dq[0].span[e[0]] - p + l0;
              const int r1 = dq[1].span[e[1]] - p + l1;
              const int r2 = d == 3 ? dq[2].span[e[2]] - p + l2 : 0;
              double* brow = &Bt[(size_t)(L.pos(k, r0, r1, r2) - off) * nb] + (ocode0 - ocode[l]);
              const double* kr = &Ke[(size_t)l * LL];
              for (int m = 0; m < LL; ++m) brow[ocode[m]] += kr[m];
            }
          }
      }
    }
  }
  // blocked transpose: a block of rows (all offsets) stays in cache while its columns are written
  constexpr int64_t kRowBlock = 256;
#pragma omp parallel for schedule(static)
  for (int64_t r0 = 0; r0 < rows; r0 += kRowBlock) {
    const int64_t r1 = std::min(rows, r0 + kRowBlock);
    for (int o = 0; o < nb; ++o) {
      double* dst = &L.band[(size_t)o * L.nloc + off];
      for (int64_t r = r0; r < r1; ++r) dst[r] = Bt[(size_t)r * nb + o];
    }
  }
}

// ---------------------------------------------------------------------------
// SIPG interface terms (Sec. 3, Eq. model:discr2):
//   -([[u]], {grad v}.n) - ([[v]], {grad u}.n) + eta ([[u]], [[v]])
// [[u]] = u_a - u_b, {w} = (w_a + w_b)/2, n the outward normal of patch a;
// quadrature on the union of both sides' breakpoints, p+1 Gauss points per
// cell and tangential direction, in the parameter of side a
// ---------------------------------------------------------------------------
namespace {
struct SideFun {
  int64_t pos;
  double val, grad[3];
};

// nonzero functions (two layers next to the side) of patch k at side point xi
void side_functions(const Problem& pr, const Level& L, int k, int side, const double* xi,
                    std::vector<SideFun>& out, double* normal, double* dS) {
  const int d = pr.d, p = pr.deg(k), P1 = p + 1;
  double X[3], J[9], Ji[9];
  geo_eval(pr, k, xi, X, J);
  const double det = inv_small(J, d, Ji);
  const int a = side / 2;
  double nrm = 0.0;
  for (int c = 0; c < d; ++c) nrm += Ji[a * d + c] * Ji[a * d + c];
  nrm = std::sqrt(nrm);
  const double sgn = side % 2 ? 1.0 : -1.0;
  for (int c = 0; c < d; ++c) normal[c] = sgn * Ji[a * d + c] / nrm;
  *dS = std::fabs(det) * nrm;
  double B[3][16], D[3][16];
  int s[3];
  for (int b = 0; b < d; ++b) {
    s[b] = find_span(L.knots[k][b], p, xi[b]);
    basis_on_span(L.knots[k][b], p, s[b], xi[b], B[b], D[b]);
  }
  out.clear();
  const int Na = L.N[k][a];
  for (int l2 = 0; l2 < (d == 3 ? P1 : 1); ++l2)
    for (int l1 = 0; l1 < P1; ++l1)
      for (int l0 = 0; l0 < P1; ++l0) {
        const int l[3] = {l0, l1, l2};
        int idx[3] = {0, 0, 0};
        for (int b = 0; b < d; ++b) idx[b] = s[b] - p + l[b];
        const int layer = side % 2 ? Na - 1 - idx[a] : idx[a];
        if (layer > 1) continue;
        SideFun f;
        f.pos = L.pos(k, idx[0], idx[1], idx[2]);
        double gh[3];
        f.val = 1.0;
        for (int b = 0; b < d; ++b) f.val *= B[b][l[b]];
        for (int c = 0; c < d; ++c) {
          gh[c] = 1.0;
          for (int b = 0; b < d; ++b) gh[c] *= (b == c) ? D[b][l[b]] : B[b][l[b]];
        }
        for (int c = 0; c < d; ++c) {
          f.grad[c] = 0.0;
          for (int b = 0; b < d; ++b) f.grad[c] += Ji[b * d + c] * gh[b];
        }
        out.push_back(f);
      }
}

Vec merged(const Vec& a, const Vec& b) {
  Vec z(a);
  z.insert(z.end(), b.begin(), b.end());
  std::sort(z.begin(), z.end());
  Vec out;
  for (double v : z)
    if (out.empty() || v - out.back() > 1e-12) out.push_back(v);
  return out;
}

double grid_size(const std::array<Vec, 3>& kn, int d) {
  double h = 0.0;
  for (int a = 0; a < d; ++a) {
    const Vec z = breakpoints(kn[a]);
    for (size_t i = 0; i + 1 < z.size(); ++i) h = std::max(h, z[i + 1] - z[i]);
  }
  return h;
}
}  // namespace

// cross: one map of cross-patch couplings per row partition (row mod cross.size()); badd: the
// within-patch terms listed per row partition (when the band is assembled elsewhere or they are
// recorded)
static void interface_terms(const Problem& pr, Level& L, const Interface& f,
                            const std::vector<std::array<Vec, 3>>& fine_knots,
                            std::vector<std::unordered_map<uint64_t, double>>& cross,
                            std::vector<std::vector<std::pair<int64_t, double>>>& badd) {
  // p: the larger degree of the two sides (Gauss points per cell exact for both sides' products)
  const int d = pr.d, p = std::max(pr.deg(f.pa), pr.deg(f.pb));
  const double eta = pr.penalty / std::min(grid_size(fine_knots[f.pa], d), grid_size(fine_knots[f.pb], d));
  const auto ta = tangential(d, f.sa), tb = tangential(d, f.sb);
  const int m = d - 1;
  const bool swap = m == 2 && (f.orient & 4u);
  // breakpoints per side-a tangential coordinate
  std::vector<Vec> cuts(m);
  for (int c = 0; c < m; ++c) {
    const int cb = swap ? 1 - c : c;
    Vec zb = breakpoints(L.knots[f.pb][tb[cb]]);
    if (f.orient & (1u << cb)) {
      Vec r(zb.size());
      for (size_t i = 0; i < zb.size(); ++i) r[i] = 1.0 - zb[zb.size() - 1 - i];
      zb = r;
    }
    cuts[c] = merged(breakpoints(L.knots[f.pa][ta[c]]), zb);
  }
  double xg[16], wg[16];
  gauss_legendre(p + 1, xg, wg);
  const int nc0 = (int)cuts[0].size() - 1, nc1 = m == 2 ? (int)cuts[1].size() - 1 : 1;
  // functions active in a cell: two normal layers times (p+1)^m tangential, per side
  int nmax = 4;
  for (int c = 0; c < m; ++c) nmax *= p + 1;
  const size_t ld = (size_t)nmax;
  // the cells' local blocks are computed in parallel (chunks of cells), then
  // added to the band / cross couplings one cell after another in cell order
  struct CellBlock {
    std::vector<int64_t> dofs;
    Vec blk;  // ld x ld
  };
  const int ncell = nc0 * nc1;
  constexpr int kCellChunk = 256;
  std::vector<CellBlock> out(std::min(ncell, kCellChunk));
  for (int cbeg = 0; cbeg < ncell; cbeg += kCellChunk) {
    const int cend = std::min(ncell, cbeg + kCellChunk);
    int too_many = 0;  // an exception must not leave the parallel region: flag it, throw after
#pragma omp parallel
    {
      std::vector<SideFun> fa, fb;
      std::unordered_map<int64_t, int> slot;
      std::vector<int> ids;
      Vec J, Dn;
#pragma omp for schedule(dynamic)
      for (int cell = cbeg; cell < cend; ++cell) {
       try {
        const int c1 = cell / nc0, c0 = cell % nc0;
        std::vector<int64_t>& dofs = out[cell - cbeg].dofs;
        Vec& blk = out[cell - cbeg].blk;
        dofs.clear();
        slot.clear();
        blk.assign(ld * ld, 0.0);
        for (int g1 = 0; g1 < (m == 2 ? p + 1 : 1); ++g1)
          for (int g0 = 0; g0 < p + 1; ++g0) {
            double s[2] = {0.0, 0.0}, w = 1.0;
            s[0] = cuts[0][c0] + (cuts[0][c0 + 1] - cuts[0][c0]) * xg[g0];
            w *= (cuts[0][c0 + 1] - cuts[0][c0]) * wg[g0];
            if (m == 2) {
              s[1] = cuts[1][c1] + (cuts[1][c1 + 1] - cuts[1][c1]) * xg[g1];
              w *= (cuts[1][c1 + 1] - cuts[1][c1]) * wg[g1];
            }
            double sb[2] = {s[0], s[1]};
            if (swap) std::swap(sb[0], sb[1]);
            for (int c = 0; c < m; ++c)
              if (f.orient & (1u << c)) sb[c] = 1.0 - sb[c];
            double xa[3] = {0, 0, 0}, xb[3] = {0, 0, 0};
            xa[f.sa / 2] = f.sa % 2 ? 1.0 : 0.0;
            xb[f.sb / 2] = f.sb % 2 ? 1.0 : 0.0;
            for (int c = 0; c < m; ++c) { xa[ta[c]] = s[c]; xb[tb[c]] = sb[c]; }
            double na[3], nb[3], dSa, dSb;
            side_functions(pr, L, f.pa, f.sa, xa, fa, na, &dSa);
            side_functions(pr, L, f.pb, f.sb, xb, fb, nb, &dSb);
            const double wq = w * dSa;
            auto reg = [&](int64_t pos) {
              auto it = slot.find(pos);
              if (it != slot.end()) return it->second;
              const int id = (int)dofs.size();
              if (id >= nmax) throw SetupError(1, "interface cell has too many active functions");
              slot.emplace(pos, id);
              dofs.push_back(pos);
              return id;
            };
            ids.clear(); J.clear(); Dn.clear();
            for (const auto& x : fa) {
              ids.push_back(reg(x.pos));
              J.push_back(x.val);
              double g = 0.0;
              for (int c = 0; c < d; ++c) g += x.grad[c] * na[c];
              Dn.push_back(0.5 * g);
            }
            for (const auto& x : fb) {
              ids.push_back(reg(x.pos));
              J.push_back(-x.val);
              double g = 0.0;
              for (int c = 0; c < d; ++c) g += x.grad[c] * na[c];
              Dn.push_back(0.5 * g);
            }
            for (size_t i = 0; i < ids.size(); ++i)
              for (size_t j = 0; j < ids.size(); ++j)
                blk[(size_t)ids[i] * ld + ids[j]] += wq * (-Dn[i] * J[j] - J[i] * Dn[j] + eta * J[i] * J[j]);
          }
       } catch (...) {
#pragma omp atomic write
        too_many = 1;
       }
      }
    }
    if (too_many) throw SetupError(1, "interface cell has too many active functions");
    // the cells' entries added in cell order; the rows are split among the threads (row mod the
    // partitions), so every entry still receives its contributions in cell order
    const int T = (int)cross.size();
    const bool list = L.band.empty() || L.record_band_add;
#pragma omp parallel num_threads(T)
    {
#pragma omp for schedule(static, 1)
      for (int t = 0; t < T; ++t)
        for (int cell = cbeg; cell < cend; ++cell) {
          const std::vector<int64_t>& dofs = out[cell - cbeg].dofs;
          const Vec& blk = out[cell - cbeg].blk;
          for (size_t i = 0; i < dofs.size(); ++i) {
            const int64_t r = dofs[i];
            if (r % T != t) continue;
            const int kr = L.patch_of[r];
            for (size_t j = 0; j < dofs.size(); ++j) {
              const double v = blk[i * ld + j];
              if (v == 0.0) continue;
              const int64_t c = dofs[j];
              const int kc = L.patch_of[c];
              if (kr == kc) {
                // same patch: inside the band (|offset| <= 1 normal, <= p tangential)
                int64_t rem_r = r - L.off[kr], rem_c = c - L.off[kc];
                int o = 0, mul = 1;
                for (int a = 0; a < d; ++a) {
                  const int ir = (int)(rem_r % L.N[kr][a]), ic = (int)(rem_c % L.N[kr][a]);
                  rem_r /= L.N[kr][a]; rem_c /= L.N[kr][a];
                  o += (ic - ir + pr.p) * mul;  // the band spans the largest degree of all patches
                  mul *= 2 * pr.p + 1;
                }
                if (list) badd[t].push_back({(int64_t)o * L.nloc + r, v});
                if (!L.band.empty()) L.band[(size_t)o * L.nloc + r] += v;
              } else {
                cross[t][((uint64_t)r << 32) | (uint64_t)c] += v;
              }
            }
          }
        }
    }
  }
}

std::vector<std::pair<int64_t, double>> Level::merged_band_add() const {
  std::vector<size_t> ord(band_add.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return band_add[a].first < band_add[b].first; });
  std::vector<std::pair<int64_t, double>> out;
  for (size_t i : ord) {
    if (!out.empty() && out.back().first == band_add[i].first) out.back().second += band_add[i].second;
    else out.push_back(band_add[i]);
  }
  return out;
}

void assemble_fine(const Problem& pr, Level& L, const std::vector<std::array<Vec, 3>>& fine_knots,
                   bool stiffness) {
  const int W = 2 * pr.p + 1;
  L.nb = pr.d == 2 ? W * W : W * W * W;
  L.band_add.clear();
  if (stiffness) {
    L.band.assign((size_t)L.nb * L.nloc, 0.0);
    for (int k = 0; k < pr.K; ++k) patch_stiffness(pr, L, k);
  } else {
    Vec().swap(L.band);
  }
  const int T = std::max(1, omp_get_max_threads());
  std::vector<std::unordered_map<uint64_t, double>> cross(T);
  std::vector<std::vector<std::pair<int64_t, double>>> badd(T);
  if (pr.coupling == 1)
    for (const auto& f : pr.ifaces) interface_terms(pr, L, f, fine_knots, cross, badd);
  // within-patch terms: the partitions one after another (a row's entries all in one partition,
  // in cell order)
  for (auto& b : badd) {
    L.band_add.insert(L.band_add.end(), b.begin(), b.end());
    std::vector<std::pair<int64_t, double>>().swap(b);
  }
  // cross-patch entries to CSR by row position: counted by row, then each row's
  // columns sorted (rows in parallel)
  std::vector<int64_t> cnt((size_t)L.nloc + 1, 0);
  size_t ncross = 0;
  for (const auto& part : cross) {
    ncross += part.size();
    for (const auto& e : part) ++cnt[(size_t)(e.first >> 32) + 1];
  }
  for (int64_t r = 0; r < L.nloc; ++r) cnt[(size_t)r + 1] += cnt[(size_t)r];
  std::vector<std::pair<int64_t, double>> ent(ncross);
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (const auto& part : cross)
      for (const auto& e : part) ent[(size_t)fill[(size_t)(e.first >> 32)]++] = {(int64_t)(e.first & 0xffffffffu), e.second};
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t r = 0; r < L.nloc; ++r)
    if (cnt[(size_t)r + 1] > cnt[(size_t)r]) std::sort(ent.begin() + cnt[(size_t)r], ent.begin() + cnt[(size_t)r + 1]);
  L.x_row.clear(); L.x_ptr.assign(1, 0); L.x_col.clear(); L.x_val.clear();
  L.x_col.reserve(ent.size());
  L.x_val.reserve(ent.size());
  for (int64_t r = 0; r < L.nloc; ++r) {
    if (cnt[(size_t)r + 1] == cnt[(size_t)r]) continue;
    L.x_row.push_back(r);
    for (int64_t q = cnt[(size_t)r]; q < cnt[(size_t)r + 1]; ++q) {
      L.x_col.push_back(ent[(size_t)q].first);
      L.x_val.push_back(ent[(size_t)q].second);
    }
    L.x_ptr.push_back((int)L.x_col.size());
  }
}

void apply_dirichlet(Level& L) {
  // offsets in parallel, the rows of one offset's column contiguous
  for (int k = 0; k < L.K && L.band.size() == (size_t)L.nb * L.nloc; ++k) {
    const int64_t r0 = L.off[k], r1 = L.off[k + 1];
#pragma omp parallel for schedule(static)
    for (int o = 0; o < L.nb; ++o) {
      const int64_t bo = L.band_offset(k, o);
      double* col = &L.band[(size_t)o * L.nloc];
      for (int64_t r = r0; r < r1; ++r) {
        if (col[r] == 0.0) continue;
        const int64_t c = r + bo;
        if (L.dirichlet[r] || c < r0 || c >= r1 || L.dirichlet[c]) col[r] = 0.0;
      }
    }
  }
  // cross blocks: drop Dirichlet rows / columns
  std::vector<int64_t> rows, cols;
  std::vector<int> ptr(1, 0);
  Vec vals;
  for (size_t i = 0; i < L.x_row.size(); ++i) {
    if (L.dirichlet[L.x_row[i]]) continue;
    const size_t before = cols.size();
    for (int j = L.x_ptr[i]; j < L.x_ptr[i + 1]; ++j)
      if (!L.dirichlet[L.x_col[j]] && L.x_val[j] != 0.0) { cols.push_back(L.x_col[j]); vals.push_back(L.x_val[j]); }
    if (cols.size() > before) { rows.push_back(L.x_row[i]); ptr.push_back((int)cols.size()); }
  }
  L.x_row.swap(rows); L.x_ptr.swap(ptr); L.x_col.swap(cols); L.x_val.swap(vals);
}

void assemble_load(const Problem& pr, const Level& L, double (*fn)(const double*, void*), void* ctx,
                   double* out) {
  const int d = pr.d;
  Vec loc(L.nloc, 0.0);
  for (int k = 0; k < pr.K; ++k) {
    const int p = pr.deg(k), P1 = p + 1, nq = p + 1;
    DirQuad dq[3];
    int ne[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) { dq[a] = dir_quad(L.knots[k][a], p); ne[a] = (int)dq[a].span.size(); }
    const int slow = d - 1;
    for (int phase = 0; phase < P1; ++phase) {
#pragma omp parallel for schedule(dynamic)
      for (int es = phase; es < ne[slow]; es += P1) {
        std::vector<double> g((size_t)nq * nq * nq);
        const int n_mid = d == 3 ? ne[1] : 1;
        for (int e1m = 0; e1m < n_mid; ++e1m)
          for (int e0 = 0; e0 < ne[0]; ++e0) {
            int e[3] = {e0, d == 2 ? es : e1m, d == 3 ? es : 0};
            for (int q2 = 0; q2 < (d == 3 ? nq : 1); ++q2)
              for (int q1 = 0; q1 < nq; ++q1)
                for (int q0 = 0; q0 < nq; ++q0) {
                  const int qi[3] = {q0, q1, q2};
                  double xi[3], w = 1.0;
                  for (int a = 0; a < d; ++a) {
                    xi[a] = dq[a].x[(size_t)e[a] * nq + qi[a]];
                    w *= dq[a].w[(size_t)e[a] * nq + qi[a]];
                  }
                  double X[3], J[9], Ji[9];
                  geo_eval(pr, k, xi, X, J);
                  const double det = inv_small(J, d, Ji);
                  g[q0 + nq * (q1 + nq * q2)] = w * std::fabs(det) * fn(X, ctx);
                }
            for (int l2 = 0; l2 < (d == 3 ? P1 : 1); ++l2)
              for (int l1 = 0; l1 < P1; ++l1)
                for (int l0 = 0; l0 < P1; ++l0) {
                  double s = 0.0;
                  for (int q2 = 0; q2 < (d == 3 ? nq : 1); ++q2)
                    for (int q1 = 0; q1 < nq; ++q1)
                      for (int q0 = 0; q0 < nq; ++q0) {
                        double b = dq[0].B[((size_t)e[0] * nq + q0) * P1 + l0] *
                                   dq[1].B[((size_t)e[1] * nq + q1) * P1 + l1];
                        if (d == 3) b *= dq[2].B[((size_t)e[2] * nq + q2) * P1 + l2];
                        s += g[q0 + nq * (q1 + nq * q2)] * b;
                      }
                  const int r0 = dq[0].span[e[0]] - p + l0, r1 = dq[1].span[e[1]] - p + l1;
                  const int r2 = d == 3 ? dq[2].span[e[2]] - p + l2 : 0;
                  loc[L.pos(k, r0, r1, r2)] += s;
                }
          }
      }
    }
  }
  for (int g = 0; g < L.ndof; ++g) out[g] = 0.0;
  for (int64_t i = 0; i < L.nloc; ++i)
    if (L.loc2glob[i] >= 0) out[L.loc2glob[i]] += loc[i];
}

}  // namespace mgiga
