// Grid hierarchy (Galerkin coarse operators), piece decomposition, fast
// diagonalisation data and the Gauss-Seidel colouring.
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <unordered_map>

#include "host.hpp"

namespace mgiga {

static std::vector<int> tangential(int d, int side) {
  std::vector<int> t;
  for (int a = 0; a < d; ++a)
    if (a != side / 2) t.push_back(a);
  return t;
}

int auto_levels(const Problem& pr) {
  const int nmin = pr.d == 2 ? 2 : 3;
  std::vector<int> counts;
  for (int k = 0; k < pr.K; ++k)
    for (int a = 0; a < pr.d; ++a) counts.push_back((int)breakpoints(pr.knots[k][a]).size() - 1);
  int levels = 1;
  for (;;) {
    bool ok = true;
    for (int n : counts) ok = ok && (n % 2 == 0) && (n / 2 >= nmin);
    if (!ok) break;
    for (int& n : counts) n /= 2;
    ++levels;
  }
  return levels;
}

// ---------------------------------------------------------------------------
// transfers: canonical embedding of nested spline spaces (Sec. 4)
// ---------------------------------------------------------------------------
Transfer build_transfer(const Level& C, const Level& F) {
  Transfer T;
  T.P.resize(F.K);
  std::map<std::pair<Vec, Vec>, Vec> cache;
  for (int k = 0; k < F.K; ++k)
    for (int a = 0; a < F.d; ++a) {
      auto key = std::make_pair(C.knots[k][a], F.knots[k][a]);
      auto it = cache.find(key);
      // (the knot vectors carry the degree through their end multiplicity, so they key the cache)
      if (it == cache.end()) it = cache.emplace(key, prolongation_1d(C.knots[k][a], F.knots[k][a], F.deg(k))).first;
      T.P[k][a] = it->second;
    }
  return T;
}

// One-direction Galerkin step of a patch band: rows and offsets in direction
// `dir` go from fine to coarse, other directions unchanged.
//   B'[(I, rest), (O, o_rest)] = sum_{i, j} P[i, I] B[(i, rest), (j - i, o_rest)] P[j, I + O]
static void coarsen_band_dir(int d, int p, const std::array<int, 3>& Nin, const Vec& Bin, int dir,
                             const Vec& P, int nc, std::array<int, 3>& Nout, Vec& Bout) {
  const int W = 2 * p + 1;
  const int nb = d == 2 ? W * W : W * W * W;
  const int nf = Nin[dir];
  Nout = Nin;
  Nout[dir] = nc;
  const int64_t rows_in = (int64_t)Nin[0] * Nin[1] * Nin[2];
  const int64_t rows_out = (int64_t)Nout[0] * Nout[1] * Nout[2];
  Bout.assign((size_t)nb * rows_out, 0.0);
  // children of each coarse index: fine i with P[i, I] != 0
  std::vector<std::vector<std::pair<int, double>>> ch(nc);
  for (int i = 0; i < nf; ++i)
    for (int I = 0; I < nc; ++I)
      if (P[(size_t)i * nc + I] != 0.0) ch[I].push_back({i, P[(size_t)i * nc + I]});
  int wpow[3] = {1, W, W * W};
  // offsets in parallel, rows innermost: the band is stored offset-major, so
  // consecutive rows read and write consecutive words of one offset's column
  const int64_t fstride[3] = {1, Nin[0], (int64_t)Nin[0] * Nin[1]};
#pragma omp parallel for schedule(dynamic)
  for (int o = 0; o < nb; ++o) {
    const int O = (o / wpow[dir]) % W - p;
    double* out = &Bout[(size_t)o * rows_out];
    int64_t r = 0;
    for (int i2 = 0; i2 < Nout[2]; ++i2)
      for (int i1 = 0; i1 < Nout[1]; ++i1)
        for (int i0 = 0; i0 < Nout[0]; ++i0, ++r) {
          const int idx[3] = {i0, i1, i2};
          const int I = idx[dir];
          const int J = I + O;
          if (J < 0 || J >= nc) continue;
          // fine row of (i, rest) without the direction's own index
          const int64_t fbase = idx[0] + fstride[1] * idx[1] + fstride[2] * idx[2] - fstride[dir] * I;
          double s = 0.0;
          for (const auto& c : ch[I]) {
            const int i = c.first;
            const int64_t frow = fbase + fstride[dir] * i;
            // the nonzeros P[j, J] are the children j of J (ascending, as the band offsets od = j - i)
            for (const auto& cj : ch[J]) {
              const int od = cj.first - i;
              if (od < -p || od > p) continue;
              const int ofine = o + (od - O) * wpow[dir];
              s += c.second * Bin[(size_t)ofine * rows_in + frow] * cj.second;
            }
          }
          out[r] = s;
        }
  }
}

void galerkin(const Level& F, const Transfer& T, Level& C, bool band) {
  const int d = F.d, p = F.p;
  C.nb = F.nb;
  if (band) C.band.assign((size_t)C.nb * C.nloc, 0.0);
  else Vec().swap(C.band);
  for (int k = 0; k < F.K && band; ++k) {
    // patch band of level F
    const int64_t rows = F.off[k + 1] - F.off[k];
    Vec B((size_t)F.nb * rows);
    for (int o = 0; o < F.nb; ++o)
      for (int64_t r = 0; r < rows; ++r) B[(size_t)o * rows + r] = F.band[(size_t)o * F.nloc + F.off[k] + r];
    std::array<int, 3> N = F.N[k];
    for (int a = 0; a < d; ++a) {
      std::array<int, 3> Nn;
      Vec Bn;
      coarsen_band_dir(d, p, N, B, a, T.P[k][a], C.N[k][a], Nn, Bn);
      N = Nn;
      B.swap(Bn);
    }
    const int64_t crow = C.off[k + 1] - C.off[k];
    for (int o = 0; o < C.nb; ++o)
      for (int64_t r = 0; r < crow; ++r) C.band[(size_t)o * C.nloc + C.off[k] + r] = B[(size_t)o * crow + r];
  }
  // cross blocks: C_c = P_a^T C P_b, tensor-product parents per direction
  auto parents = [&](int64_t pos, std::vector<std::pair<int64_t, double>>& out) {
    out.clear();
    const int k = F.patch_of[pos];
    int64_t rem = pos - F.off[k];
    int idx[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) { idx[a] = (int)(rem % F.N[k][a]); rem /= F.N[k][a]; }
    std::vector<std::pair<int, double>> par[3];
    for (int a = 0; a < 3; ++a) {
      if (a >= d) { par[a].push_back({0, 1.0}); continue; }
      const int nc = C.N[k][a];
      for (int I = 0; I < nc; ++I) {
        const double v = T.P[k][a][(size_t)idx[a] * nc + I];
        if (v != 0.0) par[a].push_back({I, v});
      }
    }
    for (const auto& x2 : par[2])
      for (const auto& x1 : par[1])
        for (const auto& x0 : par[0])
          out.push_back({C.pos(k, x0.first, x1.first, x2.first), x0.second * x1.second * x2.second});
  };
  // parents of every fine position in the couplings, once
  std::unordered_map<int64_t, int> pid;
  std::vector<int64_t> plist;
  auto want = [&](int64_t pos) {
    if (pid.emplace(pos, (int)plist.size()).second) plist.push_back(pos);
  };
  for (size_t i = 0; i < F.x_row.size(); ++i) {
    want(F.x_row[i]);
    for (int j = F.x_ptr[i]; j < F.x_ptr[i + 1]; ++j) want(F.x_col[j]);
  }
  std::vector<std::vector<std::pair<int64_t, double>>> par_of(plist.size());
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t t = 0; t < (int64_t)plist.size(); ++t) parents(plist[t], par_of[t]);
  std::vector<int> colp(F.x_col.size());
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < (int64_t)F.x_col.size(); ++j) colp[j] = pid.at(F.x_col[j]);
  // coarse rows, each with its fine coupling rows (ascending) and the row parent's weight
  std::map<int64_t, std::vector<std::pair<int, double>>> rows_of;
  for (size_t i = 0; i < F.x_row.size(); ++i)
    for (const auto& a : par_of[pid.at(F.x_row[i])]) rows_of[a.first].push_back({(int)i, a.second});
  std::vector<int64_t> crow;
  std::vector<const std::vector<std::pair<int, double>>*> cfine;
  for (const auto& e : rows_of) {
    crow.push_back(e.first);
    cfine.push_back(&e.second);
  }
  // row by row (in parallel): a coarse entry gets its contributions in the order of
  // (fine row, coupling, column parent), each as row weight * value * column weight
  std::vector<std::vector<std::pair<int64_t, double>>> res(crow.size());
#pragma omp parallel
  {
    std::vector<double> acc((size_t)C.nloc, 0.0);
    std::vector<char> mark((size_t)C.nloc, 0);
    std::vector<int64_t> touched;
#pragma omp for schedule(dynamic, 16)
    for (int64_t r = 0; r < (int64_t)crow.size(); ++r) {
      touched.clear();
      for (const auto& fi : *cfine[r]) {
        const int i = fi.first;
        const double wa = fi.second;
        for (int j = F.x_ptr[i]; j < F.x_ptr[i + 1]; ++j)
          for (const auto& b : par_of[colp[j]]) {
            if (!mark[b.first]) {
              mark[b.first] = 1;
              touched.push_back(b.first);
            }
            acc[b.first] += wa * F.x_val[j] * b.second;
          }
      }
      std::sort(touched.begin(), touched.end());
      auto& out = res[r];
      out.reserve(touched.size());
      for (int64_t c : touched) {
        out.push_back({c, acc[c]});
        acc[c] = 0.0;
        mark[c] = 0;
      }
    }
  }
  C.x_row.clear(); C.x_ptr.assign(1, 0); C.x_col.clear(); C.x_val.clear();
  for (size_t r = 0; r < crow.size(); ++r) {
    if (res[r].empty()) continue;
    C.x_row.push_back(crow[r]);
    for (const auto& e : res[r]) {
      C.x_col.push_back(e.first);
      C.x_val.push_back(e.second);
    }
    C.x_ptr.push_back((int)C.x_col.size());
  }
}

// ---------------------------------------------------------------------------
// pieces (Sec. 5, Fig. decomp): patch interiors and interface entities
// ---------------------------------------------------------------------------
std::vector<Piece> decompose(const Problem& pr, const Level& L) {
  const int d = pr.d, K = pr.K;
  // entity key: per direction 0 (start), 1 (end), 2 (free), base 3
  auto key_of = [&](const int* v) { int k = 0, m = 1; for (int a = 0; a < d; ++a) { k += v[a] * m; m *= 3; } return k; };
  const int NK = d == 2 ? 9 : 27;
  std::vector<int> par(K * NK);
  for (size_t i = 0; i < par.size(); ++i) par[i] = (int)i;
  std::function<int(int)> find = [&](int x) { while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; } return x; };
  auto unite = [&](int a, int b) { a = find(a); b = find(b); if (a != b) { if (a < b) par[b] = a; else par[a] = b; } };
  for (const auto& f : pr.ifaces) {
    const auto ta = tangential(d, f.sa), tb = tangential(d, f.sb);
    const int m = d - 1;
    const bool swap = m == 2 && (f.orient & 4u);
    const int combos = m == 1 ? 3 : 9;
    for (int cmb = 0; cmb < combos; ++cmb) {
      int va[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
      va[f.sa / 2] = f.sa % 2;
      vb[f.sb / 2] = f.sb % 2;
      int rem = cmb;
      for (int c = 0; c < m; ++c) {
        const int v = rem % 3;
        rem /= 3;
        va[ta[c]] = v;
        const int cb = swap ? 1 - c : c;
        vb[tb[cb]] = v == 2 ? 2 : (v ^ ((f.orient >> cb) & 1u ? 1 : 0));
      }
      unite(f.pa * NK + key_of(va), f.pb * NK + key_of(vb));
    }
  }
  std::vector<Piece> interior;
  std::map<int, std::vector<int>> groups;
  for (int k = 0; k < K; ++k) {
    Piece pc;
    pc.kind = 0;
    pc.patch = k;
    const auto& N = L.N[k];
    for (int64_t pos = L.off[k]; pos < L.off[k + 1]; ++pos) {
      const int g = L.loc2glob[pos];
      if (g < 0) continue;
      int64_t rem = pos - L.off[k];
      int v[3] = {2, 2, 2};
      bool inner = true;
      for (int a = 0; a < d; ++a) {
        const int i = (int)(rem % N[a]);
        rem /= N[a];
        if (i == 0) { v[a] = 0; inner = false; }
        else if (i == N[a] - 1) { v[a] = 1; inner = false; }
      }
      if (inner) pc.dofs.push_back(g);
      else groups[find(k * NK + key_of(v))].push_back(g);
    }
    std::sort(pc.dofs.begin(), pc.dofs.end());
    if (!pc.dofs.empty()) interior.push_back(pc);
  }
  std::vector<Piece> iface;
  for (auto& gr : groups) {
    Piece pc;
    pc.kind = 1;
    pc.patch = -1;
    pc.dofs = gr.second;
    std::sort(pc.dofs.begin(), pc.dofs.end());
    pc.dofs.erase(std::unique(pc.dofs.begin(), pc.dofs.end()), pc.dofs.end());
    iface.push_back(pc);
  }
  std::sort(iface.begin(), iface.end(), [](const Piece& a, const Piece& b) { return a.dofs[0] < b.dofs[0]; });
  interior.insert(interior.end(), iface.begin(), iface.end());
  return interior;
}

// ---------------------------------------------------------------------------
// fast diagonalisation of the interior operator
//   sum_a M^ x .. K^_a .. x M^ + sigma M^ x .. x M^, sigma = 1/(delta h^2)
// ---------------------------------------------------------------------------
FDData fd_setup(const Level& L, int k, double delta) {
  FDData fd;
  double h = 0.0;
  for (int a = 0; a < L.d; ++a) {
    const Vec z = breakpoints(L.knots[k][a]);
    for (size_t i = 0; i + 1 < z.size(); ++i) h = std::max(h, z[i + 1] - z[i]);
  }
  fd.sigma = 1.0 / (delta * h * h);
  for (int a = 0; a < L.d; ++a) {
    Vec Kf, Mf;
    param_matrices(L.knots[k][a], L.deg(k), Kf, Mf);
    const int N = L.N[k][a], n = N - 2;
    fd.n[a] = n;
    Vec Ki((size_t)n * n), Mi((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        Ki[(size_t)i * n + j] = Kf[(size_t)(i + 1) * N + (j + 1)];
        Mi[(size_t)i * n + j] = Mf[(size_t)(i + 1) * N + (j + 1)];
      }
    gen_eig(Ki, Mi, n, fd.U[a], fd.lam[a]);
  }
  return fd;
}

Vec restrict_dense(const Level& L, const std::vector<int>& dofs) {
  const int n = (int)dofs.size();
  std::unordered_map<int, int> local;
  for (int i = 0; i < n; ++i) local[dofs[i]] = i;
  // copies of shared DoFs
  std::unordered_map<int, int> cls;
  for (size_t c = 0; c + 1 < L.sh_ptr.size(); ++c) cls[L.loc2glob[L.sh_pos[L.sh_ptr[c]]]] = (int)c;
  std::unordered_map<int64_t, int> xrow;
  for (size_t i = 0; i < L.x_row.size(); ++i) xrow[L.x_row[i]] = (int)i;
  Vec A((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    std::vector<int64_t> copies;
    auto it = cls.find(dofs[i]);
    if (it == cls.end()) copies.push_back(L.owner[dofs[i]]);
    else for (int c = L.sh_ptr[it->second]; c < L.sh_ptr[it->second + 1]; ++c) copies.push_back(L.sh_pos[c]);
    for (int64_t pos : copies) {
      const int k = L.patch_of[pos];
      for (int o = 0; o < L.nb; ++o) {
        const double v = L.band[(size_t)o * L.nloc + pos];
        if (v == 0.0) continue;
        const int64_t c = pos + L.band_offset(k, o);
        const auto jt = local.find(L.loc2glob[c]);
        if (jt != local.end()) A[(size_t)i * n + jt->second] += v;
      }
      const auto xr = xrow.find(pos);
      if (xr != xrow.end())
        for (int j = L.x_ptr[xr->second]; j < L.x_ptr[xr->second + 1]; ++j) {
          const auto jt = local.find(L.loc2glob[L.x_col[j]]);
          if (jt != local.end()) A[(size_t)i * n + jt->second] += L.x_val[j];
        }
    }
  }
  return A;
}

// ---------------------------------------------------------------------------
// multicolour ordering for Gauss-Seidel
// ---------------------------------------------------------------------------
std::vector<int> patch_parity(const Problem& pr) {
  std::vector<std::vector<int>> nb(pr.K);
  for (const auto& f : pr.ifaces) { nb[f.pa].push_back(f.pb); nb[f.pb].push_back(f.pa); }
  for (auto& v : nb) { std::sort(v.begin(), v.end()); v.erase(std::unique(v.begin(), v.end()), v.end()); }
  std::vector<int> par(pr.K, -1);
  for (int s = 0; s < pr.K; ++s) {
    if (par[s] >= 0) continue;
    par[s] = 0;
    std::vector<int> queue{s};
    for (size_t h = 0; h < queue.size(); ++h) {
      const int cur = queue[h];
      for (int x : nb[cur])
        if (par[x] < 0) { par[x] = 1 - par[cur]; queue.push_back(x); }
    }
  }
  return par;
}

// neighbours of global DoF g (structural couplings), appended to out
static void structural_neighbours(const Problem& pr, const Level& L, int g,
                                  const std::vector<std::vector<int64_t>>& copies_of,
                                  const std::vector<std::vector<int>>& iface_nb, std::vector<int>& out) {
  const int d = L.d;
  for (int64_t pos : copies_of[g]) {
    const int k = L.patch_of[pos];
    const int p = L.deg(k);  // the patch's own reach
    int64_t rem = pos - L.off[k];
    int idx[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) { idx[a] = (int)(rem % L.N[k][a]); rem /= L.N[k][a]; }
    const int lo2 = d == 3 ? -p : 0, hi2 = d == 3 ? p : 0;
    for (int o2 = lo2; o2 <= hi2; ++o2)
      for (int o1 = -p; o1 <= p; ++o1)
        for (int o0 = -p; o0 <= p; ++o0) {
          const int j0 = idx[0] + o0, j1 = idx[1] + o1, j2 = idx[2] + o2;
          if (j0 < 0 || j0 >= L.N[k][0] || j1 < 0 || j1 >= L.N[k][1]) continue;
          if (d == 3 && (j2 < 0 || j2 >= L.N[k][2])) continue;
          const int h = L.loc2glob[L.pos(k, j0, j1, j2)];
          if (h >= 0) out.push_back(h);
        }
  }
  for (int h : iface_nb[g]) out.push_back(h);
}

std::vector<int> colouring(const Problem& pr, const Level& L) {
  // base colours modulo the largest degree + 1: a patch of lower degree couples over fewer indices
  const int d = L.d, p = L.p;
  const auto par = patch_parity(pr);
  int pw = 1;
  for (int a = 0; a < d; ++a) pw *= p + 1;
  std::vector<int> base(L.ndof);
  std::vector<std::vector<int64_t>> copies_of(L.ndof);
  for (int64_t pos = 0; pos < L.nloc; ++pos)
    if (L.loc2glob[pos] >= 0) copies_of[L.loc2glob[pos]].push_back(pos);
  for (int g = 0; g < L.ndof; ++g) {
    const int64_t pos = L.owner[g];
    const int k = L.patch_of[pos];
    int64_t rem = pos - L.off[k];
    int c = par[k] * pw, m = 1;
    for (int a = 0; a < d; ++a) {
      const int i = (int)(rem % L.N[k][a]);
      rem /= L.N[k][a];
      c += (i % (p + 1)) * m;
      m *= p + 1;
    }
    base[g] = c;
  }
  // SIPG couplings across interfaces: two layers on each side whose
  // tangential supports overlap on a set of positive measure
  std::vector<std::vector<int>> iface_nb(L.ndof);
  if (pr.coupling == 1) {
    for (const auto& f : pr.ifaces) {
      const auto ta = tangential(d, f.sa), tb = tangential(d, f.sb);
      const bool swap = d == 3 && (f.orient & 4u);
      auto layer_dofs = [&](int k, int side, std::vector<int64_t>& pos) {
        const auto& N = L.N[k];
        const int a = side / 2;
        for (int64_t q = L.off[k]; q < L.off[k + 1]; ++q) {
          int64_t rem = q - L.off[k];
          int idx[3] = {0, 0, 0};
          for (int b = 0; b < d; ++b) { idx[b] = (int)(rem % N[b]); rem /= N[b]; }
          const int layer = side % 2 ? N[a] - 1 - idx[a] : idx[a];
          if (layer <= 1) pos.push_back(q);
        }
      };
      std::vector<int64_t> pa, pb;
      layer_dofs(f.pa, f.sa, pa);
      layer_dofs(f.pb, f.sb, pb);
      auto tidx = [&](int64_t q, int k, int dir) {
        int64_t rem = q - L.off[k];
        int idx[3] = {0, 0, 0};
        for (int b = 0; b < d; ++b) { idx[b] = (int)(rem % L.N[k][b]); rem /= L.N[k][b]; }
        return idx[dir];
      };
      for (int64_t qa : pa) {
        const int ga = L.loc2glob[qa];
        if (ga < 0) continue;
        for (int64_t qb : pb) {
          const int gb = L.loc2glob[qb];
          if (gb < 0) continue;
          bool ok = true;
          for (int c = 0; c < d - 1 && ok; ++c) {
            const int cb = swap ? 1 - c : c;
            const Vec& tka = L.knots[f.pa][ta[c]];
            const Vec& tkb = L.knots[f.pb][tb[cb]];
            const int ia = tidx(qa, f.pa, ta[c]), ib = tidx(qb, f.pb, tb[cb]);
            const double lo_a = tka[ia], hi_a = tka[ia + L.deg(f.pa) + 1];
            double lo_b = tkb[ib], hi_b = tkb[ib + L.deg(f.pb) + 1];
            if ((f.orient >> cb) & 1u) { const double t = lo_b; lo_b = 1.0 - hi_b; hi_b = 1.0 - t; }
            const double lo = std::max(lo_a, lo_b), hi = std::min(hi_a, hi_b);
            ok = hi - lo > 1e-12;
          }
          if (ok) { iface_nb[ga].push_back(gb); iface_nb[gb].push_back(ga); }
        }
      }
    }
  }
  // moved: a coupled DoF of lower index with the same base colour, a coupled
  // DoF owned by another patch of the same parity, or copies in several
  // patches (conforming interface DoFs): DoFs on base colours stay inside one
  // patch and patches of one parity stay uncoupled, so patches can be swept
  // side by side
  std::vector<int> owner_patch(L.ndof);
  for (int g = 0; g < L.ndof; ++g) owner_patch[g] = L.patch_of[L.owner[g]];
  std::vector<uint8_t> moved(L.ndof, 0);
  std::vector<int> nbr;
  for (int g = 0; g < L.ndof; ++g) {
    nbr.clear();
    structural_neighbours(pr, L, g, copies_of, iface_nb, nbr);
    const int kg = owner_patch[g];
    if (copies_of[g].size() > 1) { moved[g] = 1; continue; }
    for (int h : nbr) {
      const int kh = owner_patch[h];
      if ((h < g && base[h] == base[g]) || (kh != kg && par[kh] == par[kg])) { moved[g] = 1; break; }
    }
  }
  std::vector<int> colour = base;
  const int first_extra = 2 * pw;
  for (int g = 0; g < L.ndof; ++g) {
    if (!moved[g]) continue;
    nbr.clear();
    structural_neighbours(pr, L, g, copies_of, iface_nb, nbr);
    std::vector<int> used;
    for (int h : nbr)
      if (moved[h] && h < g) used.push_back(colour[h]);
    int c = first_extra;
    while (std::find(used.begin(), used.end(), c) != used.end()) ++c;
    colour[g] = c;
  }
  return colour;
}

}  // namespace mgiga
