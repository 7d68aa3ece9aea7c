// Kernel instantiations for slices of 8 limbs per lane.
#include "kernels.cuh"

namespace mpd {
namespace {
const KernelSet set_g1 = Launch<8, 1>::make();
}  // namespace

const KernelSet* kernel_set_w8(int G) {
  switch (G) {
    case 1: return &set_g1;
    default: return nullptr;
  }
}
}  // namespace mpd
