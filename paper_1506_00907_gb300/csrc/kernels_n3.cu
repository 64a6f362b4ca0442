// Kernels of order N=3.
#define RIDG_ORDER 3
#include "instantiate.cuh"
