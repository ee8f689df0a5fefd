// Head and queue kernels for accumulators of 10 limbs (W <= 320 bits).
#define BBP_LMAX 10
#include "bbp_inst.cuh"
