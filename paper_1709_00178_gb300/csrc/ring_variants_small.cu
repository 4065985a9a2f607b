// Staged ring-kernel variants for the small rings R_{2,3} and R_{2,5} (GF(4), GF(16)).
#include "ring_kernel.cuh"

#define PYRIT_VARIANT_LIST(X) \
  X(3, 2, 8, 2, 0, 8) X(3, 1, 4, 2, 0, 16) X(5, 2, 4, 2, 0, 8) X(5, 1, 2, 2, 0, 16) X(5, 1, 4, 2, 0, 16) \
      X(5, 1, 2, 4, 0, 8) X(5, 2, 4, 1, 0, 16) X(5, 2, 8, 1, 0, 8)
#define PYRIT_VARIANT_TABLE variants_small
#include "ring_variants.inc"
