// Kernel instantiations for slices of 4 limbs per lane.
#include "kernels.cuh"

namespace mpd {
namespace {
const KernelSet set_g1 = Launch<4, 1>::make();
}  // namespace

const KernelSet* kernel_set_w4(int G) {
  switch (G) {
    case 1: return &set_g1;
    default: return nullptr;
  }
}
}  // namespace mpd
