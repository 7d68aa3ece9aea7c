// Kernel instantiation: 16 limbs per lane, 8 lanes per number (n = 128); the pivot uses the narrowest slices.
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w16_g8() {
  static const KernelSet s = Launch<16, 8>::make_with_pivot<4, 32>();
  return &s;
}
}  // namespace mpd
