// Compiled lattice shapes, complex float (mixed precision), 18^3 - 24^3 boxes.
#include "internal.cuh"
WSLDA_INSTANCE(float, 18, 18, 18, 1, 224, 1, 1, 1)
WSLDA_INSTANCE(float, 18, 18, 18, 2, 256, 1, 1, 1, 2)
WSLDA_INSTANCE(float, 18, 18, 18, 3, 192, 1, 1, 1, 3)
WSLDA_INSTANCE(float, 18, 18, 18, 3, 128, 1, 1, 1, 4)
WSLDA_INSTANCE(float, 20, 20, 20, 2, 416, 1, 1, 1)
WSLDA_INSTANCE(float, 20, 20, 20, 2, 256, 1, 1, 1, 2)
WSLDA_INSTANCE(float, 20, 20, 20, 4, 160, 1, 1, 1, 4)
WSLDA_INSTANCE(float, 24, 24, 24, 2, 288, 1, 1, 1)
WSLDA_INSTANCE(float, 24, 24, 24, 3, 256, 1, 1, 1, 2)
WSLDA_INSTANCE(float, 24, 24, 24, 4, 192, 1, 1, 1, 3)
