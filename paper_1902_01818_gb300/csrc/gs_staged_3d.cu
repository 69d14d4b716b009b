// Instances of the patch-parallel Gauss-Seidel phase for 3D patches.
#include "gs_staged.cuh"

namespace mgiga {
namespace dev {

void* gs_staged_ptr_3d(int p, int tpr) { return gs_staged_ptr_dim<3>(p, tpr); }

}  // namespace dev
}  // namespace mgiga
