// IMAD-engine Schur update with 32 limbs per lane for n = 256 and 512 limbs
// (p = 8192, 16384); see updwide_a.cu.
#include "kernels.cuh"

namespace mpd {
UpdateFn update_wide_b(int n, int minb) {
  switch (n) {
    case 256: return minb == 3 ? &Launch<32, 8>::update<3> : &Launch<32, 8>::update<4>;
    case 512: return minb == 3 ? &Launch<32, 16>::update<3> : &Launch<32, 16>::update<4>;
    default: return nullptr;
  }
}
}  // namespace mpd
