// The adjoint kernel with 16 and 32 lanes per cell.
#include "launchers.cuh"

namespace rk {
template int launch_adjoint<16>(const AdjointParams&, size_t, cudaStream_t);
template int launch_adjoint<32>(const AdjointParams&, size_t, cudaStream_t);
}  // namespace rk
