// One-warp-per-cell ROK4E variants: the tensor-core nu^T q (precision 4) and
// the mixed-precision levels 1 and 2.
#include "launchers.cuh"

namespace rk {
template int launch_rok4e<32, false, true>(const IntegrateLaunch&);
template int launch_rok4e<32, true, false>(const IntegrateLaunch&);
}  // namespace rk
