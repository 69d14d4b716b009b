// Import and validation of the C problem statement (patches, knot vectors,
// degree, geometry control points, interface pairing, SIPG penalty; Sec. 2-3)
// into the host representation of the set-up.
#include <algorithm>
#include <cstdint>

#include "host_problem.hpp"

namespace mgiga {

void import_problem(const mgiga_problem* P, Problem& pr) {
  if (!P) throw SetupError(MGIGA_EINVAL, "problem is NULL");
  if (P->dim != 2 && P->dim != 3) throw SetupError(MGIGA_EINVAL, "dim must be 2 or 3");
  if (P->num_patches < 1) throw SetupError(MGIGA_EINVAL, "num_patches must be >= 1");
  if (P->degree < 1 || P->degree > 8) throw SetupError(MGIGA_EINVAL, "degree must be in 1..8");
  if (P->geo_degree < 1 || P->geo_degree > 8) throw SetupError(MGIGA_EINVAL, "geo_degree must be in 1..8");
  if (!P->num_knots || !P->knots || !P->geo_num_knots || !P->geo_knots || !P->geo_ctrl)
    throw SetupError(MGIGA_EINVAL, "NULL array in problem");
  if (P->num_interfaces > 0 && !P->interfaces) throw SetupError(MGIGA_EINVAL, "interfaces is NULL");
  if (P->coupling != MGIGA_CONFORMING && P->coupling != MGIGA_SIPG) throw SetupError(MGIGA_EINVAL, "bad coupling");
  if (P->coupling == MGIGA_SIPG && !(P->sipg_penalty > 0.0)) throw SetupError(MGIGA_EINVAL, "sipg_penalty must be > 0");
  pr.d = P->dim;
  pr.K = P->num_patches;
  pr.p = P->degree;
  pr.pk.assign(pr.K, P->degree);
  if (P->degrees) {  // one degree per patch: degree must be the largest
    int mx = 0;
    for (int k = 0; k < pr.K; ++k) {
      if (P->degrees[k] < 1 || P->degrees[k] > 8) throw SetupError(MGIGA_EINVAL, "degrees[k] must be in 1..8");
      pr.pk[k] = P->degrees[k];
      mx = std::max(mx, P->degrees[k]);
    }
    if (mx != P->degree) throw SetupError(MGIGA_EINVAL, "degree must be the largest of degrees[]");
  }
  pr.coupling = P->coupling;
  pr.penalty = P->sipg_penalty;
  pr.knots.assign(pr.K, {});
  pr.geo.assign(pr.K, Geometry{});
  size_t kk = 0, gk = 0, gc = 0;
  for (int k = 0; k < pr.K; ++k) {
    int64_t ncp = 1;
    const int pk = pr.pk[k];
    for (int a = 0; a < pr.d; ++a) {
      const int n = P->num_knots[k * pr.d + a];
      if (n < 2 * pk + 2) throw SetupError(MGIGA_EINVAL, "knot vector too short");
      Vec t(P->knots + kk, P->knots + kk + n);
      kk += n;
      for (int i = 0; i + 1 < n; ++i)
        if (!(t[i] <= t[i + 1])) throw SetupError(MGIGA_EINVAL, "knot vector not nondecreasing");
      for (int i = 0; i <= pk; ++i)
        if (t[i] != 0.0 || t[n - 1 - i] != 1.0)
          throw SetupError(MGIGA_EINVAL, "knot vectors must be open on [0, 1] (end multiplicity p+1)");
      for (int i = pk + 1; i + 1 < n - pk - 1; ++i)
        if (t[i] == t[i + 1]) throw SetupError(MGIGA_EINVAL, "interior knots must be simple (maximal smoothness)");
      pr.knots[k][a] = t;
      const int gn = P->geo_num_knots[k * pr.d + a];
      if (gn < 2 * P->geo_degree + 2) throw SetupError(MGIGA_EINVAL, "geometry knot vector too short");
      pr.geo[k].knots[a] = Vec(P->geo_knots + gk, P->geo_knots + gk + gn);
      gk += gn;
      pr.geo[k].ncp[a] = gn - P->geo_degree - 1;
      ncp *= pr.geo[k].ncp[a];
    }
    pr.geo[k].q = P->geo_degree;
    pr.geo[k].ctrl = Vec(P->geo_ctrl + gc, P->geo_ctrl + gc + ncp * pr.d);
    gc += ncp * pr.d;
  }
  for (int i = 0; i < P->num_interfaces; ++i) {
    const mgiga_interface& f = P->interfaces[i];
    if (f.patch_a < 0 || f.patch_a >= pr.K || f.patch_b < 0 || f.patch_b >= pr.K || f.patch_a == f.patch_b)
      throw SetupError(MGIGA_EINVAL, "bad interface patch");
    if (f.side_a < 0 || f.side_a >= 2 * pr.d || f.side_b < 0 || f.side_b >= 2 * pr.d)
      throw SetupError(MGIGA_EINVAL, "bad interface side");
    if (f.orient > (pr.d == 3 ? 7u : 1u)) throw SetupError(MGIGA_EINVAL, "bad interface orientation");
    if (P->coupling == MGIGA_CONFORMING && pr.pk[f.patch_a] != pr.pk[f.patch_b])
      throw SetupError(MGIGA_EINVAL, "conforming coupling needs the same degree on both sides of an interface");
    pr.ifaces.push_back({f.patch_a, f.side_a, f.patch_b, f.side_b, f.orient});
  }
}

void init_levels(const Problem& pr, int lv, std::vector<Level>& L) {
  L.assign(lv, Level{});
  L[lv - 1].knots = pr.knots;
  for (int l = lv - 1; l > 0; --l) {
    L[l - 1].knots.resize(pr.K);
    for (int k = 0; k < pr.K; ++k)
      for (int a = 0; a < pr.d; ++a) L[l - 1].knots[k][a] = coarsen_knots(L[l].knots[k][a], pr.deg(k));
  }
  for (int l = 0; l < lv; ++l) build_topology(pr, L[l]);
}

void assemble_finest(const Problem& pr, std::vector<Level>& L) {
  Level& F = L.back();
  assemble_fine(pr, F, pr.knots);
  apply_dirichlet(F);
}

void galerkin_hierarchy(std::vector<Level>& L, std::vector<Transfer>& T) {
  const int lv = (int)L.size();
  T.assign(lv, Transfer{});
  for (int l = lv - 1; l > 0; --l) {
    T[l] = build_transfer(L[l - 1], L[l]);
    galerkin(L[l], T[l], L[l - 1]);
    apply_dirichlet(L[l - 1]);
  }
}

}  // namespace mgiga
