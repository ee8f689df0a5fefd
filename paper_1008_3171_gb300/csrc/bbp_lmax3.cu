// Head and queue kernels for accumulators of 3 limbs (W <= 96 bits).
#define BBP_LMAX 3
#include "bbp_inst.cuh"
