// Kernel instantiation: 32 limbs per lane, 32 lanes per number (n = 1024).
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w32_g32() {
  static const KernelSet s = Launch<32, 32>::make();
  return &s;
}
}  // namespace mpd
