// Head and queue kernels for accumulators of 40 limbs (W <= 1280 bits).
#define BBP_LMAX 40
#include "bbp_inst.cuh"
