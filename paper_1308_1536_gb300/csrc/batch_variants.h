// Lane geometries of the persistent batch kernel that the batch autotuner
// chooses from (internal; not part of the public ABI).  Every variant runs
// the same rounded operations on the same number layout, so results do not
// depend on the choice; only the speed does.
#pragma once
#include "kernelset.h"

namespace mpd {

struct BatchVariant {
  int W, G;    // Schur update and multipliers: W limbs per lane, G lanes per number
  int PW, PG;  // pivot phase
  cudaError_t (*launch)(MpArr X, MpArr D, MpArr Z, const BatchDescHost& bd, int p, int blocks, cudaStream_t st);
  int (*blocks_per_sm)();
};

// Variants for n limbs; entry 0 is the kernel set's own batch kernel.
// Returns the count (>= 1 for every supported n).
int batch_variants(int n, const BatchVariant** out);

// extra geometries, one translation unit per limb count
const BatchVariant* batch_variants_n16(int* count);
const BatchVariant* batch_variants_n32(int* count);
const BatchVariant* batch_variants_n64(int* count);
const BatchVariant* batch_variants_n128(int* count);

}  // namespace mpd
