// Kernel instantiation: 4 limbs per lane, 1 lanes per number (n = 4).
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w4_g1() {
  static const KernelSet s = Launch<4, 1>::make();
  return &s;
}
}  // namespace mpd
