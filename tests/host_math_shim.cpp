// Test-only C wrappers around the library's host numerics (B-spline matrices,
// knot insertion, quadrature, SPD inverse, generalised eigenproblem), compiled
// with the library's host_spline.cpp into a small shared object so that the
// CPU tests can check them against numpy/scipy and the oracle.
#include <cstring>
#include <vector>

#include "host.hpp"

using mgiga::Vec;

extern "C" {

int hm_find_span(const double* t, int nt, int p, double x) { return mgiga::find_span(Vec(t, t + nt), p, x); }

int hm_gauss(int m, double* x, double* w) {
  mgiga::gauss_legendre(m, x, w);
  return 0;
}

int hm_param_matrices(const double* t, int nt, int p, double* K, double* M) {
  try {
    Vec k, m;
    mgiga::param_matrices(Vec(t, t + nt), p, k, m);
    std::memcpy(K, k.data(), k.size() * sizeof(double));
    std::memcpy(M, m.data(), m.size() * sizeof(double));
    return 0;
  } catch (...) {
    return 1;
  }
}

int hm_prolongation(const double* tc, int ntc, const double* tf, int ntf, int p, double* P) {
  try {
    const Vec q = mgiga::prolongation_1d(Vec(tc, tc + ntc), Vec(tf, tf + ntf), p);
    std::memcpy(P, q.data(), q.size() * sizeof(double));
    return 0;
  } catch (...) {
    return 1;
  }
}

int hm_spd_inverse(const double* A, int n, int par, double* X) {
  try {
    const Vec x = mgiga::spd_inverse(Vec(A, A + (size_t)n * n), n, par != 0);
    std::memcpy(X, x.data(), x.size() * sizeof(double));
    return 0;
  } catch (const mgiga::SetupError& e) {
    return e.status;
  }
}

int hm_gen_eig(const double* K, const double* M, int n, double* U, double* lam) {
  try {
    Vec u, l;
    mgiga::gen_eig(Vec(K, K + (size_t)n * n), Vec(M, M + (size_t)n * n), n, u, l);
    std::memcpy(U, u.data(), u.size() * sizeof(double));
    std::memcpy(lam, l.data(), l.size() * sizeof(double));
    return 0;
  } catch (const mgiga::SetupError& e) {
    return e.status;
  }
}

}  // extern "C"
