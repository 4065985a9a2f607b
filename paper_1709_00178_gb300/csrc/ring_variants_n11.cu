// Staged ring-kernel variants for R_{2,11} (GF(2^10)).
#include "ring_kernel.cuh"

#define PYRIT_VARIANT_LIST(X) \
  X(11, 2, 2, 2, 0) X(11, 2, 4, 1, 0) X(11, 2, 2, 2, 1) X(11, 1, 4, 2, 0) X(11, 1, 4, 2, 1) X(11, 1, 4, 3, 0)
#define PYRIT_VARIANT_TABLE variants_n11
#include "ring_variants.inc"
