// Kernel instantiation: 8 limbs per lane, 1 lanes per number (n = 8).
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w8_g1() {
  static const KernelSet s = Launch<8, 1>::make();
  return &s;
}
}  // namespace mpd
