// Compiled lattice shapes, complex float (mixed precision), small cubes.
// WSLDA_INSTANCE(real, NX, NY, NZ, cluster size, threads, lanes per x / y / z pencil)
#include "internal.cuh"
WSLDA_INSTANCE(float, 8, 8, 8, 1, 128, 1, 1, 1)
WSLDA_INSTANCE(float, 12, 12, 12, 1, 288, 1, 1, 1)
WSLDA_INSTANCE(float, 12, 12, 12, 1, 160, 1, 1, 1, 4)
WSLDA_INSTANCE(float, 12, 12, 12, 1, 128, 1, 1, 1, 6)
WSLDA_INSTANCE(float, 16, 16, 16, 1, 256, 1, 1, 1)
WSLDA_INSTANCE(float, 16, 16, 16, 1, 256, 1, 1, 1, 2)
WSLDA_INSTANCE(float, 16, 16, 16, 2, 256, 1, 1, 1, 2)
WSLDA_INSTANCE(float, 16, 16, 16, 2, 128, 1, 1, 1, 4)
WSLDA_INSTANCE(float, 8, 12, 16, 1, 128, 1, 1, 1)
