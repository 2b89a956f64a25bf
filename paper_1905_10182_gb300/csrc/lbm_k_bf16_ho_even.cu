// Kernel instantiation, __nv_bfloat16 population storage: even-parity step of the second-order Hermite
// truncation models (M4, M5).
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(__nv_bfloat16, false, true)
