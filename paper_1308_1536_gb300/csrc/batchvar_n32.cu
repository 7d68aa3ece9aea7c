// Extra lane geometries of the batch kernel for n = 32 limbs (the batch
// autotuner's candidates beside the kernel set's own).
#include "kernels.cuh"
#include "batch_variants.h"

namespace mpd {
const BatchVariant* batch_variants_n32(int* count) {
  static const BatchVariant v[] = {
      {8, 4, 4, 8, &Launch<8, 4>::batch_p<4, 8>, &Launch<8, 4>::batch_blocks_per_sm_p<4, 8>},
      {4, 8, 4, 8, &Launch<4, 8>::batch_p<4, 8>, &Launch<4, 8>::batch_blocks_per_sm_p<4, 8>},
      {32, 1, 4, 8, &Launch<32, 1>::batch_p<4, 8>, &Launch<32, 1>::batch_blocks_per_sm_p<4, 8>},
  };
  *count = (int)(sizeof v / sizeof v[0]);
  return v;
}
}  // namespace mpd
