// ROK4E with 8 lanes per cell (FP64 and mixed precision) and the explicit
// Dormand-Prince integrator at every lane count.
#include "launchers.cuh"

namespace rk {
template int launch_rok4e<8, false, false>(const IntegrateLaunch&);
template int launch_rok4e<8, true, false>(const IntegrateLaunch&);
template int launch_rkdp<8>(const IntegrateLaunch&);
template int launch_rkdp<16>(const IntegrateLaunch&);
template int launch_rkdp<32>(const IntegrateLaunch&);
}  // namespace rk
