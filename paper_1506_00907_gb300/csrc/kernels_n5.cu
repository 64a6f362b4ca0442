// Kernels of order N=5.
#define RIDG_ORDER 5
#include "instantiate.cuh"
