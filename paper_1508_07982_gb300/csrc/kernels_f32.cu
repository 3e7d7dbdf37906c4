// Kernel instantiations for float PDF storage (float collision arithmetic).
#include "kernels_impl.cuh"

namespace lbm {
const Launchers& launchers_f32() { return LaunchImpl<float, float>::get(); }
}  // namespace lbm
