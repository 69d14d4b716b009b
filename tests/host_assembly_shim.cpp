// Test-only C wrappers around the library's host set-up (problem import, level
// layouts and numbering, quadrature assembly of the finest operator, Galerkin
// hierarchy), compiled with the library's host sources into a small shared
// object so that the CPU tests can compare the operators with the oracle's.
#include <cstdint>
#include <exception>
#include <string>
#include <vector>

#include "host_problem.hpp"

using namespace mgiga;

namespace {
struct Hierarchy {
  Problem pr;
  std::vector<Level> L;
  std::vector<Transfer> T;
};
thread_local std::string g_err;

// (row, column, value) of the global operator of level l: every copy's band
// row (conforming copies of one DoF add up) and the cross-patch couplings
template <class F>
void for_each_entry(const Level& L, F&& emit) {
  for (int64_t pos = 0; pos < L.nloc; ++pos) {
    const int g = L.loc2glob[pos];
    if (g < 0) continue;
    const int k = L.patch_of[pos];
    for (int o = 0; o < L.nb; ++o) {
      const double v = L.band[(size_t)o * L.nloc + pos];
      if (v == 0.0) continue;
      const int gc = L.loc2glob[pos + L.band_offset(k, o)];
      if (gc >= 0) emit(g, gc, v);
    }
  }
  for (size_t i = 0; i < L.x_row.size(); ++i) {
    const int g = L.loc2glob[L.x_row[i]];
    if (g < 0) continue;
    for (int j = L.x_ptr[i]; j < L.x_ptr[i + 1]; ++j) {
      const int gc = L.loc2glob[L.x_col[j]];
      if (gc >= 0) emit(g, gc, L.x_val[j]);
    }
  }
}
}  // namespace

extern "C" {

void* ha_build(const mgiga_problem* P, int levels) {
  try {
    Hierarchy* h = new Hierarchy();
    try {
      import_problem(P, h->pr);
      init_levels(h->pr, levels > 0 ? levels : auto_levels(h->pr), h->L);
      assemble_finest(h->pr, h->L);
      galerkin_hierarchy(h->L, h->T);
    } catch (...) {
      delete h;
      throw;
    }
    return h;
  } catch (const std::exception& e) {
    g_err = e.what();
    return nullptr;
  }
}

const char* ha_error() { return g_err.c_str(); }

int ha_levels(void* h) { return (int)static_cast<Hierarchy*>(h)->L.size(); }

int ha_ndof(void* h, int l) { return static_cast<Hierarchy*>(h)->L[l].ndof; }

long long ha_count(void* h, int l) {
  long long n = 0;
  for_each_entry(static_cast<Hierarchy*>(h)->L[l], [&](int, int, double) { ++n; });
  return n;
}

void ha_coo(void* h, int l, int* rows, int* cols, double* vals) {
  long long n = 0;
  for_each_entry(static_cast<Hierarchy*>(h)->L[l], [&](int r, int c, double v) {
    rows[n] = r;
    cols[n] = c;
    vals[n] = v;
    ++n;
  });
}

void ha_free(void* h) { delete static_cast<Hierarchy*>(h); }

}  // extern "C"
