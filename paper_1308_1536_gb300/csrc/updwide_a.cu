// IMAD-engine Schur update with 32 limbs per lane for n = 64 and 128 limbs
// (p = 2048, 4096): the wide lane geometry the update tuner can choose
// instead of the kernel set's own 16 limbs per lane.  Same number layout,
// same rounded operations.
#include "kernels.cuh"

namespace mpd {
UpdateFn update_wide_a(int n, int minb) {
  switch (n) {
    case 64: return minb == 3 ? &Launch<32, 2>::update<3> : &Launch<32, 2>::update<4>;
    case 128: return minb == 3 ? &Launch<32, 4>::update<3> : &Launch<32, 4>::update<4>;
    default: return nullptr;
  }
}
}  // namespace mpd
