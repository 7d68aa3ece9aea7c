// Kernel instantiation: 16 limbs per lane, 2 lanes per number (n = 32); the pivot uses the narrowest slices.
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w16_g2() {
  static const KernelSet s = Launch<16, 2>::make_with_pivot<4, 8>();
  return &s;
}
}  // namespace mpd
