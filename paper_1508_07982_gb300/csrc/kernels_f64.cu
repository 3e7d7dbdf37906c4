// Kernel instantiations for double PDF storage (double collision arithmetic).
#include "kernels_impl.cuh"

namespace lbm {
const Launchers& launchers_f64() { return LaunchImpl<double, double>::get(); }
}  // namespace lbm
