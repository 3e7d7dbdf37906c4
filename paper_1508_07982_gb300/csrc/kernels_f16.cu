// Kernel instantiations for __half PDF storage (float collision arithmetic).
#include "kernels_impl.cuh"

namespace lbm {
const Launchers& launchers_f16() { return LaunchImpl<__half, float>::get(); }
}  // namespace lbm
