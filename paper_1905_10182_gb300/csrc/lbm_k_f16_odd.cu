// Kernel instantiation, __half population storage: odd-parity step.
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(__half, true, false)
