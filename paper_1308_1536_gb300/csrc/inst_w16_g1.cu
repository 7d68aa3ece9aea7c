// Kernel instantiation: 16 limbs per lane, 1 lanes per number (n = 16); the pivot uses the narrowest slices.
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w16_g1() {
  static const KernelSet s = Launch<16, 1>::make_with_pivot<4, 4>();
  return &s;
}
}  // namespace mpd
