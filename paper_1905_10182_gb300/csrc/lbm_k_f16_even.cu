// Kernel instantiation, __half population storage: even-parity step and the auxiliary kernels.
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(__half, false, false)
CMLBM_INSTANTIATE_MISC(__half)
