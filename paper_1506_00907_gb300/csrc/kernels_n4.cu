// Kernels of order N=4.
#define RIDG_ORDER 4
#include "instantiate.cuh"
