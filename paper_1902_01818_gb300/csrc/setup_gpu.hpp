// Set-up of the level operators on the GPU (setup_gpu.cu).
#pragma once

#include <cuda_runtime.h>

#include "host.hpp"

namespace mgiga {
namespace dev {

// degrees and dimensions the device assembly covers (else the host assembles)
bool gpu_setup_supported(const Problem& pr);
// finest level: band (F.nb x F.nloc doubles, device) = patch stiffness + F.band_add (the SIPG terms
// within one patch, consumed), Dirichlet rows and columns zeroed; returns after the stream drained
void gpu_assemble_finest(const Problem& pr, Level& F, double* band, cudaStream_t st);
// cband = the patch bands of P^T A_F P (Galerkin, one direction at a time), Dirichlet rows and
// columns of C zeroed; fband, cband: device bands of F and C
void gpu_galerkin_band(const Level& F, const Level& C, const Transfer& T, const double* fband, double* cband,
                       cudaStream_t st);

}  // namespace dev
}  // namespace mgiga
