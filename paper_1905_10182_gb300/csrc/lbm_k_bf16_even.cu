// Kernel instantiation, __nv_bfloat16 population storage: even-parity step and the auxiliary kernels.
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(__nv_bfloat16, false, false)
CMLBM_INSTANTIATE_MISC(__nv_bfloat16)
