// Compiled lattice shapes, complex double (plain FP64 path).
#include "internal.cuh"
WSLDA_INSTANCE(double, 8, 8, 8, 1, 128, 1, 1, 1)
WSLDA_INSTANCE(double, 12, 12, 12, 1, 288, 1, 1, 1)
WSLDA_INSTANCE(double, 16, 16, 16, 2, 256, 1, 1, 1)
WSLDA_INSTANCE(double, 8, 12, 16, 1, 128, 1, 1, 1)
