// Kernel instantiation, __nv_bfloat16 population storage: odd-parity step.
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(__nv_bfloat16, true, false)
