// ROK4E with 16 lanes per cell (two cells per warp), FP64 and mixed precision.
#include "launchers.cuh"

namespace rk {
template int launch_rok4e<16, false, false>(const IntegrateLaunch&);
template int launch_rok4e<16, true, false>(const IntegrateLaunch&);
}  // namespace rk
