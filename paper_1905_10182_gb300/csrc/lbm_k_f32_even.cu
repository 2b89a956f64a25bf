// Kernel instantiation, float population storage: even-parity step and the auxiliary kernels.
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(float, false, false)
CMLBM_INSTANTIATE_MISC(float)
