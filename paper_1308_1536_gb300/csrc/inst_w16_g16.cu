// Kernel instantiation: 16 limbs per lane, 16 lanes per number (n = 256); the pivot uses the narrowest slices.
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w16_g16() {
  static const KernelSet s = Launch<16, 16>::make_with_pivot<8, 32>();
  return &s;
}
}  // namespace mpd
