// Head and queue kernels for accumulators of 6 limbs (W <= 192 bits).
#define BBP_LMAX 6
#include "bbp_inst.cuh"
