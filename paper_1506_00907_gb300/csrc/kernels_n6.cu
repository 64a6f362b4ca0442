// Kernels of order N=6.
#define RIDG_ORDER 6
#include "instantiate.cuh"
