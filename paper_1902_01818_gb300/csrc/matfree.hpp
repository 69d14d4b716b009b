// Matrix-free residual of the finest level by sum factorisation (matfree.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "device.cuh"
#include "host.hpp"

namespace mgiga {
namespace dev {

// one patch of the matrix-free residual: its layout, elements, tiles of elements and the offsets of
// its point tables, control points and window partials
struct MfPatch {
  int64_t off;   // first position of the patch (local layout)
  int64_t q0[3]; // first point of direction a in the point tables
  int64_t pbase; // first window partial of the patch's tiles
  int64_t ctrl;  // first control-point value (GM^d points of d values, zero padded)
  int N[3];      // B-splines per direction
  int ne[3];     // elements per direction
  int nt[3];     // tiles per direction
  int tile0;     // first CTA (tile) of the patch
};

// host-side tables (double; converted to the arithmetic type when uploaded)
struct MfHost {
  std::vector<MfPatch> pp;
  std::vector<double> B, Dv, w, gB, gD, ctrl;
  int GM = 2;           // geometry basis functions per direction in the tables (degree + 1, >= 2)
  int te = 0;           // elements per tile direction
  int ntile = 0;        // CTAs of one application
  int64_t part_n = 0;   // window partials of one application
  double flops = 0.0;   // arithmetic of one application (2 per FMA)
};

// device copies (owned by the handle)
struct MfDev {
  const MfPatch* pp = nullptr;
  int K = 0, GM = 2, ntile = 0;
  const void* B = nullptr;
  const void* Dv = nullptr;
  const void* w = nullptr;
  const void* gB = nullptr;
  const void* gD = nullptr;
  const void* ctrl = nullptr;
  const unsigned char* dir = nullptr;
  void* part = nullptr;
};

// whether the matrix-free residual covers the problem (why not, otherwise)
bool mf_supported(const Problem& pr, std::string* why);
// elements per tile direction of the kernel for (d, p, arithmetic)
int mf_tile_elems(int d, int p, bool f32);
// the point tables and tiling of the finest level F
MfHost mf_build_host(const Problem& pr, const Level& F, bool f32);
// out = f - (patch stiffness) u on the positions of `tiles` (Dirichlet rows: out = f); the SIPG
// couplings and the conforming sums are the caller's
void mf_launch(int d, int p, bool f32, const MfDev& m, cudaStream_t st, const double* u, const double* f, double* out,
               int ntiles, const Tile* tiles);

}  // namespace dev
}  // namespace mgiga
