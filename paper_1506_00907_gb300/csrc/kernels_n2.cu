// Kernels of order N=2.
#define RIDG_ORDER 2
#include "instantiate.cuh"
