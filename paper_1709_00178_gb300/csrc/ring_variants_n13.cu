// Staged ring-kernel variants for R_{2,13} (GF(2^12)).
#include "ring_kernel.cuh"

#define PYRIT_VARIANT_LIST(X) \
  X(13, 4, 1, 1, 0, 12) X(13, 2, 2, 1, 0, 16) X(13, 4, 1, 1, 0, 8) X(13, 4, 1, 1, 0, 15) X(13, 2, 2, 1, 0, 12) \
      X(13, 1, 2, 1, 0, 24) X(13, 2, 2, 1, 2, 16) X(13, 4, 1, 1, 2, 12) X(13, 4, 1, 1, 1, 12) X(13, 2, 2, 2, 0, 8) X(13, 1, 4, 2, 0, 8) X(13, 2, 1, 3, 0, 8)
#define PYRIT_VARIANT_TABLE variants_n13
#include "ring_variants.inc"
