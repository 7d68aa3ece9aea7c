// Kernel instantiation: 16 limbs per lane, 4 lanes per number (n = 64); the pivot uses the narrowest slices.
#include "kernels.cuh"

namespace mpd {
const KernelSet* kernel_set_w16_g4() {
  static const KernelSet s = Launch<16, 4>::make_with_pivot<4, 16>();
  return &s;
}
}  // namespace mpd
