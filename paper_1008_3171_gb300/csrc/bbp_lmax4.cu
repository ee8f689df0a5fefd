// Head and queue kernels for accumulators of 4 limbs (W <= 128 bits).
#define BBP_LMAX 4
#include "bbp_inst.cuh"
