// Head and queue kernels for accumulators of 16 limbs (W <= 512 bits).
#define BBP_LMAX 16
#include "bbp_inst.cuh"
