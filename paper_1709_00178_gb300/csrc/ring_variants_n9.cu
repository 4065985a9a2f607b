// Staged ring-kernel variants for R_{2,9} (GF(2^6) from the equally spaced polynomial x^6+x^3+1).
#include "ring_kernel.cuh"

#define PYRIT_VARIANT_LIST(X) \
  X(9, 4, 1, 1, 0, 12) X(9, 2, 2, 1, 0, 16) X(9, 4, 1, 1, 0, 8) X(9, 2, 4, 1, 0, 12) X(9, 2, 2, 1, 2, 16) \
      X(9, 4, 1, 1, 2, 12) X(9, 1, 4, 2, 0, 8) X(9, 1, 8, 1, 0, 12)
#define PYRIT_VARIANT_TABLE variants_n9
#include "ring_variants.inc"
