// Compiled lattice shapes, complex double, large boxes (32^3 on clusters of 16).
#include "internal.cuh"
WSLDA_INSTANCE(double, 24, 24, 24, 4, 288, 2, 2, 2)
WSLDA_INSTANCE(double, 32, 32, 32, 16, 256, 2, 2, 2)
WSLDA_INSTANCE(double, 32, 32, 32, 16, 256, 4, 4, 4, 2)
WSLDA_INSTANCE(double, 32, 32, 32, 8, 512, 4, 4, 4)
WSLDA_INSTANCE(double, 12, 12, 48, 2, 288, 1, 1, 4)
