// Kernel instantiations for slices of 16 limbs per lane.
#include "kernels.cuh"

namespace mpd {
namespace {
const KernelSet set_g1 = Launch<16, 1>::make();
const KernelSet set_g2 = Launch<16, 2>::make();
const KernelSet set_g4 = Launch<16, 4>::make();
const KernelSet set_g8 = Launch<16, 8>::make();
const KernelSet set_g16 = Launch<16, 16>::make();
const KernelSet set_g32 = Launch<16, 32>::make();
}  // namespace

const KernelSet* kernel_set_w16(int G) {
  switch (G) {
    case 1: return &set_g1;
    case 2: return &set_g2;
    case 4: return &set_g4;
    case 8: return &set_g8;
    case 16: return &set_g16;
    case 32: return &set_g32;
    default: return nullptr;
  }
}
}  // namespace mpd
