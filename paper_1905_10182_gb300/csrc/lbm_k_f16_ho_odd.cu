// Kernel instantiation, __half population storage: odd-parity step of the second-order Hermite
// truncation models (M4, M5).
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(__half, true, true)
