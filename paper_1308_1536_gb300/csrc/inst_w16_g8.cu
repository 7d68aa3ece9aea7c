// Kernel instantiation: 16 limbs per lane, 8 lanes per number (n = 128).
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w16_g8() {
  static const KernelSet s = Launch<16, 8>::make();
  return &s;
}
}  // namespace mpd
