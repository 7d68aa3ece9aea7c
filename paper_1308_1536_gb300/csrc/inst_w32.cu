// Kernel instantiations for slices of 32 limbs per lane.
#include "kernels.cuh"

namespace mpd {
namespace {
const KernelSet set_g32 = Launch<32, 32>::make();
}  // namespace

const KernelSet* kernel_set_w32(int G) {
  switch (G) {
    case 32: return &set_g32;
    default: return nullptr;
  }
}
}  // namespace mpd
