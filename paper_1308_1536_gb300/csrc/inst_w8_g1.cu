// Kernel instantiation: 8 limbs per lane, 1 lanes per number (n = 8); the pivot uses the narrowest slices.
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w8_g1() {
  static const KernelSet s = Launch<8, 1>::make_with_pivot<4, 2>();
  return &s;
}
}  // namespace mpd
