// Head and queue kernels for accumulators of 24 limbs (W <= 768 bits).
#define BBP_LMAX 24
#include "bbp_inst.cuh"
