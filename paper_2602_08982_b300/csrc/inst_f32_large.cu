// Compiled lattice shapes, complex float (mixed precision), large boxes:
// 32^3 on clusters of 4-16 (launch variants chosen by the autotuner at start),
// elongated traps 12x12x48 and 24x24x96.
#include "internal.cuh"
WSLDA_INSTANCE(float, 32, 32, 32, 8, 256, 1, 1, 1, 2)
WSLDA_INSTANCE(float, 32, 32, 32, 16, 128, 1, 1, 1, 4)
WSLDA_INSTANCE(float, 32, 32, 32, 4, 512, 1, 1, 1, 1)
WSLDA_INSTANCE(float, 32, 32, 32, 8, 256, 1, 1, 1, 3)
WSLDA_INSTANCE(float, 32, 32, 32, 8, 128, 1, 1, 1, 3)
WSLDA_INSTANCE(float, 32, 32, 32, 8, 192, 1, 1, 1, 3)
WSLDA_INSTANCE(float, 12, 12, 48, 1, 288, 1, 1, 2)
WSLDA_INSTANCE(float, 24, 24, 96, 8, 288, 1, 1, 4)
WSLDA_INSTANCE(float, 24, 24, 96, 12, 256, 1, 1, 4, 2)
WSLDA_INSTANCE(float, 24, 24, 96, 12, 192, 1, 1, 4, 3)
WSLDA_INSTANCE(float, 24, 24, 96, 12, 384, 1, 1, 4, 2)
