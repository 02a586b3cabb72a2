// Compiled lattice shapes, complex float (mixed precision), large boxes:
// 32^3 on clusters of 8, elongated traps 12x12x48 and 24x24x96.
#include "internal.cuh"
WSLDA_INSTANCE(float, 32, 32, 32, 8, 256, 1, 1, 1)
WSLDA_INSTANCE(float, 12, 12, 48, 1, 288, 1, 1, 2)
WSLDA_INSTANCE(float, 24, 24, 96, 8, 288, 1, 1, 4)
