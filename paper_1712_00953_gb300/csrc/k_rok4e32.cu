// The FP64 one-warp-per-cell ROK4E integration kernel (the default path).
#include "launchers.cuh"

namespace rk {
template int launch_rok4e<32, false, false>(const IntegrateLaunch&);
}  // namespace rk
