// Kernels of order N=1.
#define RIDG_ORDER 1
#include "instantiate.cuh"
