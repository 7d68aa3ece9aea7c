// Extra lane geometries of the batch kernel for n = 128 limbs (the batch
// autotuner's candidates beside the kernel set's own).
#include "kernels.cuh"
#include "batch_variants.h"

namespace mpd {
const BatchVariant* batch_variants_n128(int* count) {
  static const BatchVariant v[] = {
      {8, 16, 4, 32, &Launch<8, 16>::batch_p<4, 32>, &Launch<8, 16>::batch_blocks_per_sm_p<4, 32>},
      {32, 4, 4, 32, &Launch<32, 4>::batch_p<4, 32>, &Launch<32, 4>::batch_blocks_per_sm_p<4, 32>},
  };
  *count = (int)(sizeof v / sizeof v[0]);
  return v;
}
}  // namespace mpd
