// Kernel instantiation, float population storage: odd-parity step.
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(float, true, false)
