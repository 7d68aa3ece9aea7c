// Extra lane geometries of the batch kernel for n = 64 limbs (the batch
// autotuner's candidates beside the kernel set's own).
#include "kernels.cuh"
#include "batch_variants.h"

namespace mpd {
const BatchVariant* batch_variants_n64(int* count) {
  static const BatchVariant v[] = {
      {8, 8, 4, 16, &Launch<8, 8>::batch_p<4, 16>, &Launch<8, 8>::batch_blocks_per_sm_p<4, 16>},
      {32, 2, 4, 16, &Launch<32, 2>::batch_p<4, 16>, &Launch<32, 2>::batch_blocks_per_sm_p<4, 16>},
  };
  *count = (int)(sizeof v / sizeof v[0]);
  return v;
}
}  // namespace mpd
