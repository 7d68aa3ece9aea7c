// Kernel instantiation: 16 limbs per lane, 32 lanes per number (n = 512).
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w16_g32() {
  static const KernelSet s = Launch<16, 32>::make();
  return &s;
}
}  // namespace mpd
