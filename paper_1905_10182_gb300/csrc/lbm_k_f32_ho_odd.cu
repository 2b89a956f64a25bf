// Kernel instantiation, float population storage: odd-parity step of the second-order Hermite
// truncation models (M4, M5).
#include "lbm_kernels.cuh"
CMLBM_INSTANTIATE_STEP(float, true, true)
