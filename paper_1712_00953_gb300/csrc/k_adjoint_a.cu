// The adjoint kernel with 4 and 8 lanes per cell.
#include "launchers.cuh"

namespace rk {
template int launch_adjoint<4>(const AdjointParams&, size_t, cudaStream_t);
template int launch_adjoint<8>(const AdjointParams&, size_t, cudaStream_t);
}  // namespace rk
